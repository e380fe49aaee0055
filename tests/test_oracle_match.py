"""Pins of the oracle's exhaustive block matching: an independent numpy brute
force on tiny images, and the closed-form matches of a noise-free repeated
tile (d = 0 exactly at multiples of the tile period)."""
import numpy as np
import pytest

from paper_2403_03488_gb300 import synth


def brute_match(g, k, step, search, n2, tau):
    """Separate numpy implementation: all windows by slicing, lexsort by (d, index)."""
    H, W = g.shape

    def grid(L):
        p = list(range(0, L - k + 1, step))
        if (L - k) % step:
            p.append(L - k)
        return p

    hs = search // 2
    win = np.lib.stride_tricks.sliding_window_view(g, (k, k))  # [H-k+1, W-k+1, k, k]
    out = []
    for y0 in grid(H):
        for x0 in grid(W):
            ref = win[y0, x0]
            ys = np.arange(max(0, y0 - hs), min(H - k, y0 + hs) + 1)
            xs = np.arange(max(0, x0 - hs), min(W - k, x0 + hs) + 1)
            Y, X = np.meshgrid(ys, xs, indexing="ij")
            Y, X = Y.ravel(), X.ravel()
            d = ((win[Y, X] - ref) ** 2).sum(axis=(1, 2)) / (k * k)
            sel = (d <= tau) & ~((Y == y0) & (X == x0))
            Y, X, d = Y[sel], X[sel], d[sel]
            o = np.lexsort((Y * W + X, d))
            lst = [y0 * W + x0] + list((Y * W + X)[o])
            ds = [0.0] + list(d[o])
            kept = len(lst)
            n = 1
            while n * 2 <= min(kept, n2):
                n *= 2
            out.append((lst[:n2], ds, kept, n))
    return out


@pytest.mark.parametrize("H,W,tau,n2", [(16, 16, 2500.0, 16), (24, 40, 2500.0, 16),
                                        (24, 40, 400.0, 32), (19, 23, 1e9, 16), (8, 8, 2500.0, 16)])
def test_match_equals_numpy_brute_force(oracle, H, W, tau, n2):
    rng = np.random.default_rng(H * 100 + W)
    g = rng.normal(128, 40, (H, W))
    p = oracle.Pass(n2=n2, tau=tau, search=39)
    m = oracle.match(g, p)
    ref = brute_match(g, 8, 3, 39, n2, tau)
    idx = m["idx"].reshape(-1, n2)
    dist = m["dist"].reshape(-1, n2 + 1)
    for r, (lst, ds, kept, n) in enumerate(ref):
        assert m["nkept"].ravel()[r] == kept
        assert m["n"].ravel()[r] == n
        np.testing.assert_array_equal(idx[r, :len(lst)], lst)
        assert np.all(idx[r, len(lst):] == -1)
        L = min(len(ds), n2 + 1)
        np.testing.assert_allclose(dist[r, :L], ds[:L], rtol=1e-12, atol=1e-9)


def test_match_small_search_window(oracle):
    rng = np.random.default_rng(5)
    g = rng.normal(100, 30, (30, 33))
    p = oracle.Pass(n2=8, tau=1e9, search=5)
    m = oracle.match(g, p)
    ref = brute_match(g, 8, 3, 5, 8, 1e9)
    for r, (lst, ds, kept, n) in enumerate(ref):
        assert m["nkept"].ravel()[r] == kept
        np.testing.assert_array_equal(m["idx"].reshape(-1, 8)[r, :len(lst)], lst)


def test_repeated_tile_matches_at_period(oracle):
    """Noise-free tiled image: every copy of the reference at a multiple of 16
    in the window has d = 0 exactly and ranks right after the reference."""
    rng = np.random.default_rng(3)
    tile = rng.uniform(0, 255, (16, 16))
    H, W = 80, 96
    g = np.tile(tile, (H // 16, W // 16))
    p = oracle.Pass(n2=16, tau=2500.0)
    m = oracle.match(g, p)
    gy, gx = oracle.grid(H), oracle.grid(W)
    for iy, y0 in enumerate(gy):
        for ix, x0 in enumerate(gx):
            copies = [y * W + x
                      for y in range(max(0, y0 - 19), min(H - 8, y0 + 19) + 1)
                      for x in range(max(0, x0 - 19), min(W - 8, x0 + 19) + 1)
                      if (y - y0) % 16 == 0 and (x - x0) % 16 == 0 and (y, x) != (y0, x0)]
            copies.sort()
            lst = m["idx"][iy, ix]
            assert lst[0] == y0 * W + x0
            c = min(len(copies), 15)
            assert list(lst[1:1 + c]) == copies[:c]
            assert np.all(m["dist"][iy, ix, :1 + c] == 0.0)
            if 1 + c < 17:
                assert m["dist"][iy, ix, 1 + c] != 0.0  # next rank is farther, or absent (-1)


def test_constant_image_ties_break_by_index(oracle):
    g = np.full((20, 20), 77.0)
    m = oracle.match(g, oracle.Pass(n2=16))
    lst = m["idx"][1, 1]  # reference at (3, 3)
    assert lst[0] == 3 * 20 + 3
    others = sorted(y * 20 + x for y in range(13) for x in range(13) if (y, x) != (3, 3))
    assert list(lst[1:]) == others[:15]
    assert m["n"][1, 1] == 16 and m["flag"].max() == 0


def test_flags_near_tau_and_ties(oracle):
    g = np.zeros((8, 9))
    g[:, 8] = 50.0  # patch at x=1 differs from x=0 by one column of 50: d = 8*2500/64
    d = 8 * 2500.0 / 64
    m = oracle.match(g, oracle.Pass(tau=d))
    assert m["flag"][0, 0] & oracle.FLAG_TAU
    m = oracle.match(g, oracle.Pass(tau=d * 1.01))
    assert m["flag"][0, 0] == 0 and m["n"][0, 0] == 2


def test_synthetic_scene_match_smoke(oracle):
    clean, noisy = synth.make_batch([0], 48, 56, 25.0)
    m = oracle.match(noisy[0, 0], oracle.Pass())
    assert m["n"].min() >= 1 and m["n"].max() <= 16
    assert np.all((m["n"] & (m["n"] - 1)) == 0)


@pytest.mark.parametrize("k,step,search,H,W,tau,n2", [(12, 4, 39, 30, 34, 5000.0, 16), (11, 6, 39, 29, 40, 3500.0, 32),
                                                      (12, 4, 9, 25, 26, 1e9, 16), (11, 6, 15, 11, 23, 3500.0, 8)])
def test_match_larger_patches_equal_numpy_brute_force(oracle, k, step, search, H, W, tau, n2):
    """The high-noise profile's 12 x 12 / step 4 and 11 x 11 / step 6 patches
    against the same independent brute force (distances / k^2)."""
    rng = np.random.default_rng(k * 1000 + H)
    g = rng.normal(128, 60, (H, W))
    p = oracle.Pass(patch=k, step=step, search=search, n2=n2, tau=tau)
    m = oracle.match(g, p)
    ref = brute_match(g, k, step, search, n2, tau)
    idx = m["idx"].reshape(-1, n2)
    dist = m["dist"].reshape(-1, n2 + 1)
    assert len(ref) == idx.shape[0]
    for r, (lst, ds, kept, n) in enumerate(ref):
        assert m["nkept"].ravel()[r] == kept
        assert m["n"].ravel()[r] == n
        np.testing.assert_array_equal(idx[r, :len(lst)], lst)
        L = min(len(ds), n2 + 1)
        np.testing.assert_allclose(dist[r, :L], ds[:L], rtol=1e-12, atol=1e-9)

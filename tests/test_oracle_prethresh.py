"""Pins of the oracle's block matching on 2D-prethresholded patches (BM3D's
first-pass distance at high noise): d(P, Q) = ||Y(P) - Y(Q)||^2 / 64 with
Y(P) = the orthonormal 2D DCT-II of P, coefficients of magnitude <= thr
zeroed.

- thr = 0 reduces to the pixel-domain matcher (the transform is orthonormal);
- a brute force written with scipy's DCT (an independent transform) and a
  full lexicographic sort agrees on every unflagged reference, for several
  thresholds and window shapes;
- a threshold above every coefficient makes all distances 0, so groups are
  the reference followed by the window in row-major order;
- a coefficient exactly at the threshold raises the PRE flag, and an empty
  band never does;
- the first pass with lambda2d and a zero noise-derived threshold equals
  the plain first pass."""
import numpy as np
import pytest
from scipy.fft import dctn

from paper_2403_03488_gb300 import synth


def brute(g, p, thr):
    g = np.asarray(g, np.float64)
    H, W = g.shape
    k = p.patch
    Hp, Wp = H - k + 1, W - k + 1
    Y = np.empty((Hp, Wp, k * k))
    for y in range(Hp):
        for x in range(Wp):
            c = dctn(g[y:y + k, x:x + k], norm="ortho").ravel()
            Y[y, x] = np.where(np.abs(c) > thr, c, 0.0)
    gy = [int(v) for v in range(0, H - k + 1, p.step)]
    gx = [int(v) for v in range(0, W - k + 1, p.step)]
    if gy[-1] != H - k:
        gy.append(H - k)
    if gx[-1] != W - k:
        gx.append(W - k)
    hs = p.search // 2
    out = {}
    for ry, y0 in enumerate(gy):
        for rx, x0 in enumerate(gx):
            cand = []
            for y in range(max(0, y0 - hs), min(H - k, y0 + hs) + 1):
                for x in range(max(0, x0 - hs), min(W - k, x0 + hs) + 1):
                    if (y, x) == (y0, x0):
                        continue
                    d = ((Y[y0, x0] - Y[y, x]) ** 2).sum() / float(k * k)
                    if d <= p.tau:
                        cand.append((d, y * W + x))
            cand.sort()
            kept = len(cand) + 1
            n = 1
            while n * 2 <= min(kept, p.n2):
                n *= 2
            out[(ry, rx)] = (n, [y0 * W + x0] + [c[1] for c in cand[:n - 1]], [0.0] + [c[0] for c in cand[:n - 1]])
    return out


def test_zero_threshold_is_the_pixel_matcher(oracle):
    _, noisy = synth.make_batch([3], 40, 48, 50.0)
    p = oracle.Pass(n2=16, tau=5000.0)
    a = oracle.match(noisy[0, 0], p)
    b = oracle.match_pre(noisy[0, 0], p, 0.0)
    np.testing.assert_array_equal(a["idx"], b["idx"])
    np.testing.assert_array_equal(a["n"], b["n"])
    np.testing.assert_allclose(b["dist"], a["dist"], rtol=1e-10, atol=1e-9)


@pytest.mark.parametrize("thr,step,search,n2,H,W", [(100.0, 3, 39, 16, 30, 27), (60.0, 3, 11, 16, 24, 24),
                                                     (250.0, 2, 9, 8, 21, 19), (40.0, 5, 15, 32, 26, 33)])
def test_brute_force_with_scipy_dct(oracle, thr, step, search, n2, H, W):
    _, noisy = synth.make_batch([5], H, W, 50.0)
    g = noisy[0, 0]
    p = oracle.Pass(step=step, search=search, n2=n2, tau=5000.0)
    om = oracle.match_pre(g, p, thr)
    bf = brute(g, p, thr)
    checked = 0
    for (ry, rx), (n, lst, dl) in bf.items():
        if om["flag"][ry, rx]:
            continue
        checked += 1
        assert om["n"][ry, rx] == n
        np.testing.assert_array_equal(om["idx"][ry, rx, :n], lst)
        np.testing.assert_allclose(om["dist"][ry, rx, :n], dl, rtol=1e-9, atol=1e-9)
    assert checked >= 0.5 * len(bf)


@pytest.mark.parametrize("thr,H,W", [(100.0, 30, 33), (40.0, 25, 29)])
def test_brute_force_with_scipy_dct_12x12_step_4(oracle, thr, H, W):
    """The high-noise profile's first pass: 12 x 12 patches on a step-4 grid."""
    _, noisy = synth.make_batch([9], H, W, 50.0)
    g = noisy[0, 0]
    p = oracle.Pass(patch=12, step=4, search=39, n2=16, tau=5000.0)
    om = oracle.match_pre(g, p, thr)
    bf = brute(g, p, thr)
    checked = 0
    for (ry, rx), (n, lst, dl) in bf.items():
        if om["flag"][ry, rx]:
            continue
        checked += 1
        assert om["n"][ry, rx] == n
        np.testing.assert_array_equal(om["idx"][ry, rx, :n], lst)
        np.testing.assert_allclose(om["dist"][ry, rx, :n], dl, rtol=1e-9, atol=1e-9)
    assert checked >= 0.5 * len(bf)


def test_threshold_above_every_coefficient(oracle):
    _, noisy = synth.make_batch([7], 20, 22, 50.0)
    g = noisy[0, 0]
    p = oracle.Pass(n2=16, tau=5000.0, search=7)
    om = oracle.match_pre(g, p, 1e9, band=0.0)
    W = g.shape[1]
    gy, gx = oracle.grid(20), oracle.grid(22)
    for ry, y0 in enumerate(gy):
        for rx, x0 in enumerate(gx):
            win = [y * W + x for y in range(max(0, y0 - 3), min(12, y0 + 3) + 1)
                   for x in range(max(0, x0 - 3), min(14, x0 + 3) + 1) if (y, x) != (y0, x0)]
            assert om["n"][ry, rx] == 16
            np.testing.assert_array_equal(om["idx"][ry, rx], [y0 * W + x0] + win[:15])
            assert np.all(om["dist"][ry, rx, :16] == 0.0)


def test_prethreshold_hazard_flag(oracle):
    g = np.full((16, 16), 40.0)  # every patch: DC = 8 * 40 = 320, all other coefficients 0
    p = oracle.Pass(n2=4, tau=5000.0, search=5)
    assert np.all(oracle.match_pre(g, p, 320.0)["flag"] & oracle.FLAG_PRE)
    assert np.all(oracle.match_pre(g, p, 320.0 + 1e-3)["flag"] & oracle.FLAG_PRE)
    assert not np.any(oracle.match_pre(g, p, 300.0)["flag"] & oracle.FLAG_PRE)
    # zero band: only an exact tie with the threshold is a hazard
    assert not np.any(oracle.match_pre(g, p, 320.5, band=0.0)["flag"] & oracle.FLAG_PRE)


def test_first_pass_with_zero_prethreshold_is_the_plain_first_pass(oracle):
    _, noisy = synth.make_batch([9], 24, 26, 50.0)
    x = noisy[0]
    a, _, _ = oracle.bm3d_pass1(x, [50.0], oracle.Pass(n2=16, tau=5000.0))
    b, _, _ = oracle.bm3d_pass1(x, [0.0 + 50.0], oracle.Pass(n2=16, tau=5000.0, lambda2d=1e-12))
    np.testing.assert_allclose(b, a, rtol=0, atol=1e-9)
    c, _, _ = oracle.bm3d_pass1(x, [50.0], oracle.Pass(n2=16, tau=5000.0, lambda2d=2.0))
    assert np.abs(c - a).max() > 1e-3  # the prethreshold changes the groups at sigma 50


def test_regime_selects_the_prethreshold_above_sigma_40(oracle):
    """Regime 0 switches to tau = 5000 / 3500 and the prethresholded first
    pass strictly above sigma = 40; regime 1 never does; the second pass never
    prethresholds."""
    for sigma, regime, lam, t1, t2 in ((40.0, 0, 0.0, 2500.0, 400.0), (40.5, 0, 2.0, 5000.0, 3500.0),
                                       (50.0, 1, 0.0, 2500.0, 400.0), (15.0, 0, 0.0, 2500.0, 400.0)):
        h, w = oracle.default_passes(sigma, regime)
        assert (h.lambda2d, h.tau, w.tau, w.lambda2d) == (lam, t1, t2, 0.0), (sigma, regime)

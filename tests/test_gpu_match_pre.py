"""Block matching on 2D-prethresholded patches (BM3D's first-pass distance at
high noise) on the GPU against the FP64 oracle, through the C ABI.

Match lists must equal the oracle's except at references the oracle flags: a
candidate tied with tau, two ranked distances tied, or a prethresholded
coefficient within 0.005 of the threshold (its keep/zero decision may go
either way in FP32) that could reach the group.  Two distances a, b are tied
when |a - b| <= 1e-5 max(a, b) + 1e-3 (sqrt(a) + sqrt(b)): the FP32
transforms leave each coefficient difference within 5e-4, which moves a
distance d by at most 1e-3 sqrt(d).  Flagged lists must still be valid
rankings, within the same tolerance, under the FP64 prethresholded distance.
The denoiser picks the path per image: sigma > 40 images of a mixed batch
give the same output as alone, and the end-to-end PSNR at sigma = 50 stays
within 0.05 dB of the oracle's BM3D with the same regime."""
import numpy as np
import pytest
from scipy.fft import dctn

from gpu_util import dev, host, need_gpu
from paper_2403_03488_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def api():
    from paper_2403_03488_gb300 import api as A
    return A


def pre_dists(guide, ref_idx, lst, thr):
    W = guide.shape[1]

    def Y(i):
        y, x = divmod(int(i), W)
        c = dctn(guide[y:y + 8, x:x + 8].astype(np.float64), norm="ortho")
        return np.where(np.abs(c) > thr, c, 0.0)

    r = Y(ref_idx)
    return np.array([((r - Y(q)) ** 2).mean() for q in lst])


def check_pre(oracle, gidx, gn, om, guide, tau, thr):
    Ry, Rx = om["n"].shape
    flagged = 0
    for ry in range(Ry):
        for rx in range(Rx):
            no, ng = int(om["n"][ry, rx]), int(gn[ry, rx])
            ol, gl = om["idx"][ry, rx], gidx[ry, rx]
            if om["flag"][ry, rx] == 0:
                assert ng == no, (ry, rx, ng, no)
                np.testing.assert_array_equal(gl[:no], ol[:no], err_msg=str((ry, rx)))
                continue
            flagged += 1
            assert gl[0] == ol[0]
            d = pre_dists(guide, gl[0], gl[1:ng], thr)
            assert np.all(d <= tau * (1 + 1e-5) + 2e-3 * np.sqrt(tau))
            assert np.all(np.diff(d) >= -(1e-5 * np.maximum(d[1:], d[:-1]) + 1e-3 * (np.sqrt(d[1:]) + np.sqrt(d[:-1]))))
    return Ry * Rx, flagged


@pytest.mark.parametrize("H,W,sigmas,n2", [(64, 72, (50.0,), 16), (37, 50, (60.0, 45.0), 16), (8, 8, (50.0,), 16),
                                           (9, 13, (50.0,), 8), (101, 67, (75.0,), 32), (70, 140, (50.0,), 16)])
def test_match_pre_parity(oracle, H, W, sigmas, n2):
    """Grids of several CTA tiles (32 x 4 references) with ragged tails, and
    degenerate one-reference images; thr = 2 sigma."""
    A = api()
    B = len(sigmas)
    _, noisy = synth.make_batch(range(40, 40 + B), H, W, list(sigmas))
    p = A.default_bm3d_params().hard
    p.n2 = n2
    thrs = [2.0 * s for s in sigmas]
    idx, n = A.bm3d_match_prethresh(dev(noisy[:, 0]), [5000.0] * B, thrs, p)
    idx, n = host(idx), host(n)
    total = flagged = 0
    for b in range(B):
        om = oracle.match_pre(noisy[b, 0], oracle.Pass(n2=n2, tau=5000.0), thrs[b])
        t, f = check_pre(oracle, idx[b], n[b], om, noisy[b, 0], 5000.0, thrs[b])
        total, flagged = total + t, flagged + f
    assert flagged <= 0.6 * total + 1, (flagged, total)  # at least 40 % checked exactly


@pytest.mark.parametrize("step,search,thr", [(4, 21, 100.0), (2, 15, 60.0), (3, 39, 0.0)])
def test_match_pre_other_steps_and_zero_threshold(oracle, step, search, thr):
    """Other grid steps and windows; thr = 0 is the pixel-domain distance
    evaluated through the transform."""
    A = api()
    _, noisy = synth.make_batch([47], 45, 58, 50.0)
    p = A.default_bm3d_params().hard
    p.step, p.search = step, search
    idx, n = A.bm3d_match_prethresh(dev(noisy[:, 0]), [2500.0], [thr], p)
    om = oracle.match_pre(noisy[0, 0], oracle.Pass(step=step, search=search, n2=16, tau=2500.0), thr)
    check_pre(oracle, host(idx)[0], host(n)[0], om, noisy[0, 0], 2500.0, thr)


def test_match_pre_wide_window_direct_row_loads(oracle):
    """A step and window wide enough (step 6, search 77: 270 staged pixels per
    row, more than the 256 the CTA prefetches) that the kernel loads each new
    pixel row directly; the image is 300 pixels wide so the staged row is not
    clipped."""
    A = api()
    _, noisy = synth.make_batch([48], 40, 300, 50.0)
    p = A.default_bm3d_params().hard
    p.step, p.search = 6, 77
    idx, n = A.bm3d_match_prethresh(dev(noisy[:, 0]), [5000.0], [100.0], p)
    om = oracle.match_pre(noisy[0, 0], oracle.Pass(step=6, search=77, n2=16, tau=5000.0), 100.0)
    t, f = check_pre(oracle, host(idx)[0], host(n)[0], om, noisy[0, 0], 5000.0, 100.0)
    assert f <= 0.6 * t + 1, (f, t)


def test_match_pre_repeated_tile_exact(oracle):
    """Exact duplicates of the reference get distance 0 (same transform
    arithmetic for reference and candidates), so lists on a periodic image
    equal the oracle's everywhere."""
    A = api()
    rng = np.random.default_rng(8)
    g = np.tile(rng.uniform(0, 255, (16, 16)), (5, 6)).astype(np.float32)
    p = A.default_bm3d_params().hard
    idx, n = A.bm3d_match_prethresh(dev(g[None]), [5000.0], [100.0], p)
    om = oracle.match_pre(g, oracle.Pass(tau=5000.0), 100.0)
    gi, gn = host(idx)[0], host(n)[0]
    for ry in range(om["n"].shape[0]):
        for rx in range(om["n"].shape[1]):
            k = om["n"][ry, rx]
            d = om["dist"][ry, rx, 1:k]
            exact = int(np.sum(d == 0.0))  # the duplicates lead the list, in index order
            if om["flag"][ry, rx] == 0:
                assert gn[ry, rx] == k
                np.testing.assert_array_equal(gi[ry, rx, :k], om["idx"][ry, rx, :k])
            np.testing.assert_array_equal(gi[ry, rx, :1 + exact], om["idx"][ry, rx, :1 + exact])


def test_mixed_batch_takes_each_path_per_image():
    """sigma > 40 images match on prethresholded patches, the others on
    pixels; every image of a mixed batch denoises exactly as it does alone."""
    A = api()
    sig = [25.0, 50.0, 15.0, 60.0, 45.0]
    _, noisy = synth.make_batch(range(60, 65), 48, 56, sig)
    x = dev(noisy)
    batch = host(A.denoise_bm3d(x, sig))
    for b, s in enumerate(sig):
        alone = host(A.denoise_bm3d(dev(noisy[b:b + 1]), [s]))
        np.testing.assert_array_equal(batch[b], alone[0])
    # regime 1 (raw patches at every sigma) differs on the high-noise images only
    q = A.default_bm3d_params()
    q.sigma_regime = 1
    raw = host(A.denoise_bm3d(x, sig, q))
    for b, s in enumerate(sig):
        assert (np.abs(raw[b] - batch[b]).max() > 0) == (s > 40), (b, s)


@pytest.mark.parametrize("C,sigma", [(1, 50.0), (3, 60.0)])
def test_denoise_high_sigma_psnr_matches_oracle(oracle, C, sigma):
    A = api()
    clean, noisy = synth.make_batch([70], 72, 80, sigma, C=C)
    g = host(A.denoise_bm3d(dev(noisy), [sigma]))[0]
    _, o = oracle.bm3d(noisy[0].astype(np.float64), sigma)
    pg, po = oracle.psnr(g, clean[0]), oracle.psnr(o, clean[0])
    assert abs(pg - po) < 0.05, (pg, po)
    # the prethresholded first pass is what the oracle's regime-0 BM3D runs at this sigma
    _, o_raw = oracle.bm3d(noisy[0].astype(np.float64), sigma, regime=1)
    assert np.abs(o - o_raw).max() > 1e-3


def test_match_pre_full_size_sampled(oracle):
    """1024 x 1024 at sigma = 50 (the size the high-noise bench runs): the
    lists of 200 sampled references against the oracle run on crops that
    contain each reference's whole search window (unflagged references exact)."""
    A = api()
    _, noisy = synth.make_batch([110, 111], 1024, 1024, 50.0)
    p = A.default_bm3d_params().hard
    idx, n = A.bm3d_match_prethresh(dev(noisy[:, 0]), [5000.0, 5000.0], [100.0, 100.0], p)
    idx, n = host(idx), host(n)
    gy = np.array(A.grid(1024))
    rng = np.random.default_rng(6)
    checked = bad = 0
    for _ in range(200):
        b = int(rng.integers(0, 2))
        ry, rx = int(rng.integers(0, len(gy))), int(rng.integers(0, len(gy)))
        y0, x0 = int(gy[ry]), int(gy[rx])
        cy, cx = (max(0, y0 - 19) // 3) * 3, (max(0, x0 - 19) // 3) * 3
        ey, ex = min(1024, y0 + 27), min(1024, x0 + 27)
        om = oracle.match_pre(noisy[b, 0, cy:ey, cx:ex], oracle.Pass(tau=5000.0), 100.0)
        oy, ox = list(oracle.grid(ey - cy)).index(y0 - cy), list(oracle.grid(ex - cx)).index(x0 - cx)
        if om["flag"][oy, ox]:
            continue
        checked += 1
        k = int(om["n"][oy, ox])
        assert n[b, ry, rx] == k
        ol = om["idx"][oy, ox, :k]
        full = (ol // (ex - cx) + cy) * 1024 + ol % (ex - cx) + cx
        bad += int(not np.array_equal(idx[b, ry, rx, :k], full))
    assert bad == 0 and checked >= 80, (bad, checked)

"""BM3D parity of the CUDA path against the FP64 oracle, stage by stage.

Match lists: exact, except references the oracle flags (a candidate within
1e-5 tau of tau, or two ranked distances within 1e-5 relative), whose lists
must still be valid rankings.  Filtering: each pass is fed the oracle's match
lists (and, for the Wiener pass, the oracle's basic estimate rounded to FP32),
so no decision cascades; pixels must agree within 1e-3 on the 0..255 scale,
except, in the hard-threshold pass, pixels covered by a group with a 3D
coefficient within 1e-3 of lambda * sigma (the FP32 coefficient error bound
derived in the design notes is below 2.5e-4).  End to end: PSNR within
0.05 dB of the oracle."""
import numpy as np
import pytest

from gpu_util import dev, footprint, host, need_gpu
from paper_2403_03488_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 1e-3
BAND = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def api():
    from paper_2403_03488_gb300 import api as A
    return A


def dists64(guide, ref_idx, lst, W):
    y0, x0 = divmod(int(ref_idx), W)
    P = guide[y0:y0 + 8, x0:x0 + 8].astype(np.float64)
    out = []
    for q in lst:
        y, x = divmod(int(q), W)
        out.append(((P - guide[y:y + 8, x:x + 8]) ** 2).mean())
    return np.array(out)


def check_match(oracle, gidx, gn, om, guide, tau):
    """Returns (#references, #flagged)."""
    Ry, Rx = om["n"].shape
    W = guide.shape[1]
    flagged = 0
    for ry in range(Ry):
        for rx in range(Rx):
            no, ng = int(om["n"][ry, rx]), int(gn[ry, rx])
            ol, gl = om["idx"][ry, rx], gidx[ry, rx]
            fl = int(om["flag"][ry, rx])
            if fl == 0:
                assert ng == no, (ry, rx, ng, no)
                np.testing.assert_array_equal(gl[:no], ol[:no], err_msg=str((ry, rx)))
                continue
            flagged += 1
            assert gl[0] == ol[0]
            d = dists64(guide, gl[0], gl[1:ng], W)
            assert np.all(d <= tau * (1 + 1e-5))
            assert np.all(np.diff(d) >= -1e-5 * np.maximum(d[1:], 1e-30))
            if not fl & oracle.FLAG_TAU:
                assert ng == no
                np.testing.assert_allclose(d, om["dist"][ry, rx, 1:ng], rtol=1e-5)
    return Ry * Rx, flagged


@pytest.mark.parametrize("H,W,sigmas", [(64, 72, (25.0,)), (37, 50, (15.0, 50.0)), (8, 8, (25.0,)),
                                        (9, 13, (25.0,)), (101, 67, (35.0,))])
def test_match_parity_hard(oracle, H, W, sigmas):
    A = api()
    B = len(sigmas)
    _, noisy = synth.make_batch(range(10, 10 + B), H, W, list(sigmas))
    taus = [5000.0 if s > 40 else 2500.0 for s in sigmas]
    p = A.default_bm3d_params().hard
    idx, n = A.bm3d_match(dev(noisy[:, 0]), taus, p)
    idx, n = host(idx), host(n)
    for b in range(B):
        om = oracle.match(noisy[b, 0], oracle.Pass(n2=16, tau=taus[b]))
        check_match(oracle, idx[b], n[b], om, noisy[b, 0], taus[b])


@pytest.mark.parametrize("step,search,n2,H,W", [(4, 39, 16, 61, 70), (2, 21, 8, 40, 37), (5, 15, 32, 33, 52),
                                                (1, 9, 4, 20, 19)])
def test_match_parity_other_steps(oracle, step, search, n2, H, W):
    """Grid steps other than 3 take the any-step kernel (register-blocked over
    8 candidates, same distance association); lists exact vs the oracle."""
    A = api()
    _, noisy = synth.make_batch([14], H, W, 25.0)
    p = A.default_bm3d_params().hard
    p.step, p.search, p.n2 = step, search, n2
    idx, n = A.bm3d_match(dev(noisy[:, 0]), [2500.0], p)
    om = oracle.match(noisy[0, 0], oracle.Pass(step=step, search=search, n2=n2, tau=2500.0))
    check_match(oracle, host(idx)[0], host(n)[0], om, noisy[0, 0], 2500.0)


@pytest.mark.parametrize("n2", [1, 2, 8, 32])
def test_match_parity_group_sizes_on_basic(oracle, n2):
    A = api()
    clean, noisy = synth.make_batch([21], 70, 61, 25.0)
    basic, _, _ = oracle.bm3d_pass1(noisy[0], [25.0], oracle.Pass())
    g = basic[0].astype(np.float32)
    p = A.default_bm3d_params().wiener
    p.n2 = n2
    idx, n = A.bm3d_match(dev(g[None]), [400.0], p)
    om = oracle.match(g, oracle.Pass(n2=n2, tau=400.0))
    check_match(oracle, host(idx)[0], host(n)[0], om, g, 400.0)


def test_match_repeated_tile_exact(oracle):
    A = api()
    rng = np.random.default_rng(3)
    g = np.tile(rng.uniform(0, 255, (16, 16)), (5, 6)).astype(np.float32)
    p = A.default_bm3d_params().hard
    idx, n = A.bm3d_match(dev(g[None]), [2500.0], p)
    om = oracle.match(g, oracle.Pass())
    np.testing.assert_array_equal(host(n)[0], om["n"])
    gi = host(idx)[0]
    for ry in range(om["n"].shape[0]):
        for rx in range(om["n"].shape[1]):
            k = om["n"][ry, rx]
            np.testing.assert_array_equal(gi[ry, rx, :k], om["idx"][ry, rx, :k])


@pytest.mark.parametrize("n2,tau", [(32, 400.0), (16, 2500.0), (32, 1e9)])
def test_match_exact_ties_in_index_order(oracle, n2, tau):
    """Pixels of 4 levels make every distance an exact multiple of 1/64 in
    FP32 as in FP64, so equal distances abound at every rank: the lists must
    equal the oracle's (ties by index) whatever order the kernel scans its
    candidates in (the 31-entry list scans rows from the centre out and
    re-matches a reference with a tie in index order)."""
    A = api()
    rng = np.random.default_rng(11)
    g = rng.integers(0, 4, (53, 67)).astype(np.float32)
    p = A.default_bm3d_params().wiener
    p.n2 = n2
    idx, n = A.bm3d_match(dev(g[None]), [tau], p)
    om = oracle.match(g, oracle.Pass(n2=n2, tau=tau))
    np.testing.assert_array_equal(host(n)[0], om["n"])
    gi = host(idx)[0]
    for ry in range(om["n"].shape[0]):
        for rx in range(om["n"].shape[1]):
            k = om["n"][ry, rx]
            np.testing.assert_array_equal(gi[ry, rx, :k], om["idx"][ry, rx, :k], err_msg=str((ry, rx)))


def test_match_constant_image_index_order(oracle):
    """All distances 0: every list is the first candidates in index order."""
    A = api()
    g = np.full((40, 45), 77.0, np.float32)
    p = A.default_bm3d_params().wiener
    idx, n = A.bm3d_match(dev(g[None]), [400.0], p)
    om = oracle.match(g, oracle.Pass(n2=32, tau=400.0))
    np.testing.assert_array_equal(host(n)[0], om["n"])
    np.testing.assert_array_equal(host(idx)[0], om["idx"])


def _ycc_or_grey(oracle, noisy):
    return noisy.astype(np.float64) if noisy.shape[1] == 1 else np.stack([oracle.rgb_to_ycc(x) for x in noisy])


@pytest.mark.parametrize("C,H,W,sigmas", [(1, 64, 80, (25.0, 15.0)), (3, 45, 52, (25.0,)), (1, 33, 91, (50.0,))])
def test_filter_hard_parity_given_oracle_matches(oracle, C, H, W, sigmas):
    A = api()
    B = len(sigmas)
    _, noisy = synth.make_batch(range(30, 30 + B), H, W, list(sigmas), C=C)
    img = _ycc_or_grey(oracle, noisy).astype(np.float32)
    hard = A.default_bm3d_params().hard
    idx, ns, ref, ok, sig_flat = [], [], [], [], []
    for b in range(B):
        sc = oracle.channel_sigmas(sigmas[b], C)
        sig_flat += list(sc)
        P = oracle.default_passes(sigmas[b])[0]
        om = oracle.pass1_matches(img[b, 0], P, sc[0])
        basic, pf, _ = oracle.bm3d_pass1(img[b], sc, P, band=BAND)
        idx.append(om["idx"])
        ns.append(om["n"])
        ref.append(basic)
        ok.append((pf & oracle.FLAG_THR) == 0)
        hard.tau = P.tau
    out = host(A.bm3d_filter_hard(dev(img), dev(np.stack(idx).astype(np.int32)), dev(np.stack(ns).astype(np.int32)),
                                  sig_flat, hard))
    for b in range(B):
        m = ok[b]
        assert m.mean() > 0.5, "too many hazard pixels: %.3f" % m.mean()
        err = np.abs(out[b] - ref[b])[:, m]
        assert err.max() <= TOL, (b, err.max())


@pytest.mark.parametrize("n2", [32, 8])
def test_filter_hard_parity_other_group_sizes(oracle, n2):
    """The first pass with groups of up to 32 patches (one group per warp)
    and of up to 8 (two groups per warp, lists loaded one pair ahead): within
    TOL of the oracle outside the hazard band."""
    A = api()
    _, noisy = synth.make_batch([33], 70, 75, 25.0)
    img = noisy.astype(np.float64).astype(np.float32)
    hard = A.default_bm3d_params().hard
    hard.n2 = n2
    sc = oracle.channel_sigmas(25.0, 1)
    P = oracle.default_passes(25.0)[0]
    P.n2 = n2
    om = oracle.pass1_matches(img[0, 0], P, sc[0])
    basic, pf, _ = oracle.bm3d_pass1(img[0], sc, P, band=BAND)
    hard.tau = P.tau
    out = host(A.bm3d_filter_hard(dev(img), dev(om["idx"][None].astype(np.int32)), dev(om["n"][None].astype(np.int32)),
                                  list(sc), hard))
    m = (pf & oracle.FLAG_THR) == 0
    assert m.mean() > 0.5, "too many hazard pixels: %.3f" % m.mean()
    err = np.abs(out[0] - basic)[:, m]
    assert err.max() <= TOL, err.max()


@pytest.mark.parametrize("C,H,W,sigma", [(1, 64, 80, 25.0), (3, 40, 57, 15.0), (1, 50, 50, 50.0)])
def test_filter_wiener_parity_given_oracle_basic(oracle, C, H, W, sigma):
    A = api()
    _, noisy = synth.make_batch([40], H, W, sigma, C=C)
    img = _ycc_or_grey(oracle, noisy).astype(np.float32)
    sc = oracle.channel_sigmas(sigma, C)
    P1, P2 = oracle.default_passes(sigma)
    basic, _, _ = oracle.bm3d_pass1(img[0], sc, P1)
    basic32 = basic.astype(np.float32)
    om = oracle.match(basic32[0], P2)
    final, _, _ = oracle.bm3d_pass2(img[0], basic32, sc, P2)
    p = A.default_bm3d_params().wiener
    p.tau = P2.tau
    out = host(A.bm3d_filter_wiener(dev(img), dev(basic32[None]), dev(om["idx"][None].astype(np.int32)),
                                    dev(om["n"][None].astype(np.int32)), list(sc), p))
    err = np.abs(out[0] - final)
    assert err.max() <= TOL, err.max()


def test_filter_parity_with_heavy_weights_and_large_values(oracle):
    """Contributions beyond the fast fixed-point range: values up to ~1000
    (the image scaled by 4, so w kai v >= 512 in the bright parts), an exact
    zero block where every 3D coefficient is thresholded (N_har = 0, weight
    sigma^2 = 10^4 after scaling), and for the Wiener pass a basic estimate
    that is 0.2 on a block (sum of squared gains ~1e-4, weight ~1e4)."""
    A = api()
    H, W, sigma = 56, 64, 100.0
    _, noisy = synth.make_batch([77], H, W, 25.0)
    img = (noisy[0] * 4.0).astype(np.float32)
    img[:, 8:32, 30:54] = 0.0
    sc = [sigma]
    P1, P2 = oracle.default_passes(sigma)
    om = oracle.pass1_matches(img[0].astype(np.float64), P1, sc[0])
    basic, pf, _ = oracle.bm3d_pass1(img.astype(np.float64), sc, P1, band=4 * BAND)
    hard = A.default_bm3d_params().hard
    hard.tau = P1.tau
    out = host(A.bm3d_filter_hard(dev(img[None]), dev(om["idx"][None].astype(np.int32)),
                                  dev(om["n"][None].astype(np.int32)), sc, hard))
    ok = (pf & oracle.FLAG_THR) == 0
    assert ok.mean() > 0.5
    assert np.abs(out[0] - basic)[:, ok].max() <= 4 * TOL
    basic32 = basic.astype(np.float32)
    basic32[:, 30:50, 4:28] = 0.2
    om2 = oracle.match(basic32[0].astype(np.float64), P2)
    final, _, _ = oracle.bm3d_pass2(img.astype(np.float64), basic32.astype(np.float64), sc, P2)
    p = A.default_bm3d_params().wiener
    p.tau = P2.tau
    out2 = host(A.bm3d_filter_wiener(dev(img[None]), dev(basic32[None]), dev(om2["idx"][None].astype(np.int32)),
                                     dev(om2["n"][None].astype(np.int32)), sc, p))
    assert np.abs(out2[0] - final).max() <= 4 * TOL


@pytest.mark.parametrize("C,H,W,sigmas", [(1, 96, 96, (25.0, 25.0)), (3, 64, 72, (25.0,)), (1, 80, 88, (50.0,))])
def test_denoise_bm3d_psnr_matches_oracle(oracle, C, H, W, sigmas):
    A = api()
    B = len(sigmas)
    clean, noisy = synth.make_batch(range(50, 50 + B), H, W, list(sigmas), C=C)
    out = host(A.denoise_bm3d(dev(noisy), list(sigmas)))
    for b in range(B):
        _, final = oracle.bm3d(noisy[b], sigmas[b])
        pg, po = oracle.psnr(out[b], clean[b]), oracle.psnr(final, clean[b])
        assert abs(pg - po) <= 0.05, (b, pg, po)
        assert pg > oracle.psnr(noisy[b], clean[b]) + 5.0


def test_constant_image_closed_form_on_gpu(oracle):
    A = api()
    img = np.full((1, 1, 40, 48), 100.0, np.float32)
    out = host(A.denoise_bm3d(dev(img), [25.0]))
    B2 = 64.0 * 32.0 * 100.0 ** 2
    np.testing.assert_allclose(out, 100.0 * B2 / (B2 + 625.0), atol=1e-3)


def test_colour_transform_parity(oracle):
    A = api()
    x = np.random.default_rng(0).uniform(0, 255, (2, 3, 17, 23)).astype(np.float32)
    y = host(A.rgb_to_ycc(dev(x)))
    for b in range(2):
        np.testing.assert_allclose(y[b], oracle.rgb_to_ycc(x[b]), atol=1e-3)
    z = host(A.ycc_to_rgb(dev(y)))
    for b in range(2):
        np.testing.assert_allclose(z[b], oracle.ycc_to_rgb(y[b].astype(np.float64)), atol=1e-3)


def test_error_reduce_fp64(oracle):
    A = api()
    rng = np.random.default_rng(1)
    ref = rng.uniform(0, 255, (3, 2, 31, 29)).astype(np.float32)
    out = (ref + rng.normal(0, 9, ref.shape)).astype(np.float32)
    sse, mx = A.error_reduce(dev(out), dev(ref))
    sse, mx = host(sse), host(mx)
    for b in range(3):
        e = np.clip(out[b].astype(np.float64), 0, 255) - ref[b]
        assert abs(sse[b] - (e * e).sum()) <= 1e-9 * (e * e).sum()
        assert mx[b] == np.abs(out[b].astype(np.float64) - ref[b]).max()
        assert abs(10 * np.log10(255 ** 2 / (sse[b] / out[b].size)) - oracle.psnr(out[b], ref[b])) < 1e-9


def test_match_full_size_sampled(oracle):
    """1024 x 1024 (the precision-path image size): the match lists of 300
    sampled references against the oracle run on crops that contain each
    reference's whole search window."""
    A = api()
    _, noisy = synth.make_batch([100, 101], 1024, 1024, 25.0)
    p = A.default_bm3d_params().hard
    idx, n = A.bm3d_match(dev(noisy[:, 0]), [2500.0, 2500.0], p)
    idx, n = host(idx), host(n)
    gy = np.array(A.grid(1024))
    rng = np.random.default_rng(5)
    bad = 0
    for _ in range(300):
        b = int(rng.integers(0, 2))
        ry, rx = int(rng.integers(0, len(gy))), int(rng.integers(0, len(gy)))
        y0, x0 = int(gy[ry]), int(gy[rx])
        cy, cx = (max(0, y0 - 19) // 3) * 3, (max(0, x0 - 19) // 3) * 3
        ey, ex = min(1024, y0 + 27), min(1024, x0 + 27)
        crop = noisy[b, 0, cy:ey, cx:ex]
        om = oracle.match(crop, oracle.Pass())
        oy, ox = list(oracle.grid(ey - cy)).index(y0 - cy), list(oracle.grid(ex - cx)).index(x0 - cx)
        k = int(om["n"][oy, ox])
        if om["flag"][oy, ox]:
            continue
        assert n[b, ry, rx] == k
        ol = om["idx"][oy, ox, :k]
        full = (ol // (ex - cx) + cy) * 1024 + ol % (ex - cx) + cx
        bad += int(not np.array_equal(idx[b, ry, rx, :k], full))
    assert bad == 0


@pytest.mark.parametrize("H,W,sigma,n2,tau,basic", [(64, 72, 25.0, 16, 2500.0, False), (101, 67, 50.0, 16, 5000.0, False),
                                                  (9, 13, 25.0, 16, 2500.0, False), (130, 97, 25.0, 32, 400.0, True),
                                                  (70, 61, 15.0, 8, 400.0, True), (40, 300, 25.0, 2, 2500.0, False)])
def test_match_tc_prefilter_equals_fp32_and_oracle(oracle, H, W, sigma, n2, tau, basic):
    """Tensor-core prefilter + exact FP32 re-rank: bit-identical match lists
    to the exhaustive FP32 kernel, and oracle parity."""
    A = api()
    _, noisy = synth.make_batch([80, 81], H, W, sigma)
    g = noisy[:, 0]
    if basic:
        g = np.stack([oracle.bm3d_pass1(noisy[b], [sigma], oracle.Pass())[0][0] for b in range(2)]).astype(np.float32)
    p = A.default_bm3d_params().hard
    p.n2 = n2
    i32, n32 = A.bm3d_match(dev(g), [tau, tau], p, precision=A.DN_FP32)
    itc, ntc = A.bm3d_match(dev(g), [tau, tau], p, precision=A.DN_BF16_MATCH)
    i32, n32, itc, ntc = host(i32), host(n32), host(itc), host(ntc)
    np.testing.assert_array_equal(ntc, n32)
    for b in range(2):
        for ry in range(n32.shape[1]):
            for rx in range(n32.shape[2]):
                k = n32[b, ry, rx]
                np.testing.assert_array_equal(itc[b, ry, rx, :k], i32[b, ry, rx, :k])
        om = oracle.match(g[b], oracle.Pass(n2=n2, tau=tau))
        check_match(oracle, itc[b], ntc[b], om, g[b], tau)
    assert A.device_error() == 0


@pytest.mark.parametrize("H,W,tx,ty", [(200, 180, 1, 1), (64, 72, 0, 0)])
def test_tc_cross_terms_within_proven_bound(H, W, tx, ty):
    """The FP16 tensor-core cross terms of a reference tile agree with the exact
    dot products of the centred patches a = P - m, b = Q - m within the bound
    the prefilter relies on: |x_hat - x| <= (2^-10 + 2^-14 + 2^-22) sum |a_i b_i|
    + 64 * 2^-25 (|a|_inf + |b|_inf) (FP16 rounding of both operands, FP32
    accumulation, subnormals), and the bound is not vacuous: the error is
    mostly far below it and above zero (the operands really are rounded)."""
    A = api()
    _, noisy = synth.make_batch([85], H, W, 25.0)
    g = noisy[0, 0]
    p = A.default_bm3d_params().hard
    cross, m, (cy0, cx0) = A.bm3d_match_cross_terms(dev(g), p, 2500.0, tx, ty)
    cross, m = host(cross), float(host(m)[0])
    gy, gx = A.grid(H), A.grid(W)
    hs = 19
    y_last = gy[min(ty * 16 + 15, len(gy) - 1)]
    x_last = gx[min(tx * 8 + 7, len(gx) - 1)]
    CH, CW = min(H - 8, y_last + hs) - cy0 + 1, min(W - 8, x_last + hs) - cx0 + 1
    g64 = g.astype(np.float64)
    checked, ratios = 0, []
    for t in range(0, 128, 7):
        ry, rx = ty * 16 + t // 8, tx * 8 + t % 8
        if ry >= len(gy) or rx >= len(gx):
            continue
        a = g64[gy[ry]:gy[ry] + 8, gx[rx]:gx[rx] + 8] - np.float32(m)
        for s in range(0, cross.shape[1] * 128, 5):
            row, col = s // 64, s % 64
            if row >= CH or col >= CW:
                continue
            b = g64[cy0 + row:cy0 + row + 8, cx0 + col:cx0 + col + 8] - np.float32(m)
            x = (a * b).sum()
            bound = (2.0 ** -10 + 2.0 ** -14 + 2.0 ** -22) * np.abs(a * b).sum() + \
                64 * 2.0 ** -25 * (np.abs(a).max() + np.abs(b).max())
            err = abs(float(cross[t, row // 2, s % 128]) - x)
            assert err <= bound, (t, row, col, cross[t, row // 2, s % 128], x)
            ratios.append(err / bound)
            checked += 1
    assert checked > 500
    assert 0.0 < np.median(ratios) < 0.5


def test_match_tc_prefilter_equals_fp32_full_size():
    """At the precision-path size (two 1024^2 images) the tensor-core prefilter
    with exact re-rank and the FP32 kernels (tiled step-3 kernel, warp kernel for
    the off-lattice row and column) give identical lists and group sizes for
    both passes: one distance association, exact ties broken by index."""
    A = api()
    _, noisy = synth.make_batch([100, 101], 1024, 1024, 25.0)
    x = dev(noisy)
    hard = A.default_bm3d_params().hard
    i32, n32 = A.bm3d_match(x[:, 0].contiguous(), [2500.0, 2500.0], hard, precision=A.DN_FP32)
    itc, ntc = A.bm3d_match(x[:, 0].contiguous(), [2500.0, 2500.0], hard, precision=A.DN_BF16_MATCH)
    assert np.array_equal(host(n32), host(ntc))
    assert np.array_equal(host(i32), host(itc))
    basic = A.bm3d_filter_hard(x, i32, n32, [25.0, 25.0], hard)
    wien = A.default_bm3d_params().wiener
    g = basic[:, 0].contiguous()
    i32, n32 = A.bm3d_match(g, [400.0, 400.0], wien, precision=A.DN_FP32)
    itc, ntc = A.bm3d_match(g, [400.0, 400.0], wien, precision=A.DN_BF16_MATCH)
    assert np.array_equal(host(n32), host(ntc))
    assert np.array_equal(host(i32), host(itc))
    assert A.device_error() == 0


def test_bm3d_with_tc_matching_equals_fp32():
    """With the tensor-core prefiltered matcher the match lists are the FP32 ones, so
    the BM3D output is bit-identical (the filtering stays FP32)."""
    A = api()
    _, noisy = synth.make_batch([90, 91], 150, 170, [25.0, 50.0])
    x = dev(noisy)
    a = host(A.denoise_bm3d(x, [25.0, 50.0], A.default_bm3d_params(precision=A.DN_FP32)))
    b = host(A.denoise_bm3d(x, [25.0, 50.0], A.default_bm3d_params(precision=A.DN_BF16_MATCH)))
    assert np.array_equal(a, b)
    assert A.device_error() == 0


def test_denoise_bm3d_is_bitwise_reproducible():
    """Aggregation sums are exact (fixed point), so repeated runs, with other
    work in between, give bit-identical outputs."""
    A = api()
    _, noisy = synth.make_batch([70, 71, 72], 200, 168, [25.0, 15.0, 50.0])
    x = dev(noisy)
    a = host(A.denoise_bm3d(x, [25.0, 15.0, 50.0]))
    A.denoise_nlm(x, 25.0)
    b = host(A.denoise_bm3d(x, [25.0, 15.0, 50.0]))
    assert np.array_equal(a, b)


def test_denoise_bm3d_full_size_properties(oracle):
    A = api()
    clean, noisy = synth.make_batch([100, 101], 1024, 1024, 25.0)
    out = host(A.denoise_bm3d(dev(noisy), 25.0))
    assert np.isfinite(out).all()
    for b in range(2):
        assert oracle.psnr(out[b], clean[b]) > oracle.psnr(noisy[b], clean[b]) + 8.0

"""BM3D with the 2D patch transforms on the tensor cores (precision DN_BF16)
against the FP64 oracle and the FP32 GPU path.

The BF16 path rounds three things to BF16 (unit roundoff 2^-8): the
mean-centred pixels of every patch, the 64 x 64 DCT matrix D and the
filtered spectra entering the inverse; the patch means (the DC terms) stay in
FP32.  Where no decision depends on the rounding, an estimate's error is
bounded through the orthonormal transform by the 2-norm of its centred patch:
|dx|_inf <= |dX|_2 <= 3 * 2^-8 * |r|_2 for the three roundings, plus one more
2^-8 |r|_2 for the rounded D not being exactly orthonormal and the sensitivity
of the Wiener gains; aggregation is a convex combination of estimates, so the
output error is at most BOUND = 4 * 2^-8 * max over patches of |r|_2.  The
hard threshold is a decision: a coefficient within the rounding of lambda
sigma can flip (about one per few groups at these sizes), which moves that
group's estimate by up to lambda sigma times a basis function.  So the hard
pass is held to the quality bar instead -- PSNR within 0.05 dB of the oracle
-- and to a mean error that such flips cannot exceed (0.01 sigma + 0.05)."""
import numpy as np
import pytest

from gpu_util import dev, host, need_gpu
from paper_2403_03488_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def api():
    from paper_2403_03488_gb300 import api as A
    return A


def bound(img):
    """4 * 2^-8 * the largest 2-norm of a mean-centred 8x8 patch of img [C][H][W]."""
    from numpy.lib.stride_tricks import sliding_window_view
    w = sliding_window_view(img.astype(np.float64), (8, 8), axis=(1, 2))
    r = w - w.mean(axis=(-1, -2), keepdims=True)
    return 4.0 * 2.0 ** -8 * np.sqrt((r * r).sum(axis=(-1, -2))).max()


def _img(oracle, noisy):
    return noisy.astype(np.float64) if noisy.shape[1] == 1 else np.stack([oracle.rgb_to_ycc(x) for x in noisy])


@pytest.mark.parametrize("C,H,W,sigma", [(1, 128, 128, 25.0), (1, 112, 120, 15.0), (1, 128, 120, 50.0),
                                         (3, 72, 80, 25.0)])
def test_filter_bf16_stagewise(oracle, C, H, W, sigma):
    """Each pass fed the oracle's match lists (pass 2 also its basic estimate):
    hard pass PSNR within 0.05 dB of the oracle and mean error within the
    flip allowance; Wiener pass within BOUND everywhere."""
    A = api()
    clean, noisy = synth.make_batch([130], H, W, sigma, C=C)
    img = _img(oracle, noisy)[0].astype(np.float32)
    cref = _img(oracle, clean)[0]
    sc = oracle.channel_sigmas(sigma, C)
    P1, P2 = oracle.default_passes(sigma)
    om = oracle.pass1_matches(img[0], P1, sc[0])
    basic, _, _ = oracle.bm3d_pass1(img, sc, P1)
    hard = A.default_bm3d_params().hard
    hard.tau = P1.tau
    out = host(A.bm3d_filter_hard(dev(img[None]), dev(om["idx"][None].astype(np.int32)),
                                  dev(om["n"][None].astype(np.int32)), list(sc), hard, precision=A.DN_BF16))[0]
    assert np.isfinite(out).all()
    assert abs(oracle.psnr(out, cref) - oracle.psnr(basic, cref)) <= 0.05
    assert np.abs(out - basic).mean() <= 0.01 * sigma + 0.05
    basic32 = basic.astype(np.float32)
    om2 = oracle.match(basic32[0], P2)
    final, _, _ = oracle.bm3d_pass2(img, basic32, sc, P2)
    p = A.default_bm3d_params().wiener
    p.tau = P2.tau
    out2 = host(A.bm3d_filter_wiener(dev(img[None]), dev(basic32[None]), dev(om2["idx"][None].astype(np.int32)),
                                     dev(om2["n"][None].astype(np.int32)), list(sc), p, precision=A.DN_BF16))[0]
    err = np.abs(out2 - final)
    assert err.max() <= bound(img), (err.max(), bound(img))
    assert err.mean() <= 0.05
    assert A.device_error() == 0


def test_filter_bf16_hard_identity_at_zero_threshold(oracle):
    """lambda3d = 0 keeps every coefficient: the pass returns its input, up to
    the BF16 rounding bound (the oracle pins the exact identity)."""
    A = api()
    _, noisy = synth.make_batch([131], 70, 90, 25.0)
    img = noisy[0].astype(np.float32)
    P1 = oracle.Pass(lambda3d=0.0)
    om = oracle.match(img[0], P1)
    hard = A.default_bm3d_params().hard
    hard.lambda3d = 0.0
    out = host(A.bm3d_filter_hard(dev(img[None]), dev(om["idx"][None].astype(np.int32)),
                                  dev(om["n"][None].astype(np.int32)), [25.0], hard, precision=A.DN_BF16))[0]
    assert np.abs(out - img).max() <= bound(img)


@pytest.mark.parametrize("C,H,W,sigmas", [(1, 128, 128, (25.0, 50.0)), (3, 96, 104, (25.0,))])
def test_denoise_bm3d_bf16_psnr(oracle, C, H, W, sigmas):
    """End to end: within 0.05 dB of the oracle and of the FP32 GPU path."""
    A = api()
    B = len(sigmas)
    clean, noisy = synth.make_batch(range(140, 140 + B), H, W, list(sigmas), C=C)
    x = dev(noisy)
    o16 = host(A.denoise_bm3d(x, list(sigmas), A.default_bm3d_params(precision=A.DN_BF16)))
    o32 = host(A.denoise_bm3d(x, list(sigmas), A.default_bm3d_params(precision=A.DN_FP32)))
    for b in range(B):
        _, ref = oracle.bm3d(noisy[b], sigmas[b])
        p16 = oracle.psnr(o16[b], clean[b])
        assert abs(p16 - oracle.psnr(ref, clean[b])) <= 0.05
        assert abs(p16 - oracle.psnr(o32[b], clean[b])) <= 0.05
    assert A.device_error() == 0


def test_bf16_constant_image_closed_form():
    """Flat patches centre to zero, so the BF16 path keeps the closed form of
    the FP32 one: hard pass identity, Wiener DC gain B^2 / (B^2 + sigma^2)."""
    A = api()
    img = np.full((1, 1, 40, 48), 100.0, np.float32)
    out = host(A.denoise_bm3d(dev(img), [25.0], A.default_bm3d_params(precision=A.DN_BF16)))
    B2 = 64.0 * 32.0 * 100.0 ** 2
    np.testing.assert_allclose(out, 100.0 * B2 / (B2 + 625.0), atol=1e-3)


@pytest.mark.parametrize("hard_n2,wiener_n2", [(32, 16), (1, 1), (8, 2)])
def test_bf16_group_slot_sizes(hard_n2, wiener_n2):
    """Groups of up to 32 patches in the hard pass and of up to 16 in the
    Wiener pass (the other slot sizes of the kernel), and tiny groups: the
    BF16 result stays within 0.05 dB of the FP32 GPU path with the same
    parameters (which the oracle pins)."""
    A = api()
    clean, noisy = synth.make_batch([150, 151], 96, 112, [25.0, 15.0])
    x = dev(noisy)
    res = []
    for prec in (A.DN_FP32, A.DN_BF16):
        p = A.default_bm3d_params(precision=prec)
        p.hard.n2, p.wiener.n2 = hard_n2, wiener_n2
        res.append(host(A.denoise_bm3d(x, [25.0, 15.0], p)))
    from oracle import psnr
    for b in range(2):
        assert abs(psnr(res[1][b], clean[b]) - psnr(res[0][b], clean[b])) <= 0.05
    assert A.device_error() == 0


def test_bf16_bitwise_reproducible_and_ragged():
    """Deterministic tensor-core results and exact aggregation: repeated
    runs are bit-identical; ragged sizes (several CTA tiles plus tails) and a
    batch that spans more images than the persistent grid has CTAs per tile."""
    A = api()
    clean, noisy = synth.make_batch([160, 161, 162], 203, 171, [25.0, 15.0, 50.0])
    x = dev(noisy)
    p = A.default_bm3d_params(precision=A.DN_BF16)
    a = host(A.denoise_bm3d(x, [25.0, 15.0, 50.0], p))
    A.denoise_nlm(x, 25.0)
    b = host(A.denoise_bm3d(x, [25.0, 15.0, 50.0], p))
    assert np.array_equal(a, b)
    from oracle import psnr
    for i in range(3):
        assert psnr(a[i], clean[i]) > psnr(noisy[i], clean[i]) + 5.0
    assert A.device_error() == 0


def test_bf16_full_size(oracle):
    """16 x 1024^2 at sigma 25 (the precision-path workload): finite, within
    0.05 dB of the FP32 GPU path on every image."""
    A = api()
    clean, noisy = synth.make_batch(list(range(100, 116)), 1024, 1024, 25.0)
    x = dev(noisy)
    o16 = host(A.denoise_bm3d(x, 25.0, A.default_bm3d_params(precision=A.DN_BF16)))
    o32 = host(A.denoise_bm3d(x, 25.0, A.default_bm3d_params(precision=A.DN_FP32)))
    assert np.isfinite(o16).all()
    for b in range(16):
        assert abs(oracle.psnr(o16[b], clean[b]) - oracle.psnr(o32[b], clean[b])) <= 0.05
    assert A.device_error() == 0

"""Pins of the oracle's BM3D passes by closed forms and special cases:
lambda3D = 0 returns the input, a huge threshold returns 0, the Wiener pass
with sigma -> 0 returns the noisy image, a constant image is a fixed point,
and a two-patch case whose result follows from scipy's DCT and numpy's
Kaiser window (it fixes the group weight 1/(sigma^2 N_har) and the window)."""
import numpy as np
import pytest
import scipy.fft

from paper_2403_03488_gb300 import synth


@pytest.mark.parametrize("C", [1, 3])
def test_lambda_zero_is_identity(oracle, C):
    _, noisy = synth.make_batch([11], 40, 44, 25.0, C=C)
    x = noisy[0].astype(np.float64)
    basic, _, _ = oracle.bm3d_pass1(x, [25.0] * C, oracle.Pass(lambda3d=0.0))
    np.testing.assert_allclose(basic, x, atol=1e-9)


def test_huge_threshold_gives_zero(oracle):
    _, noisy = synth.make_batch([12], 32, 32, 25.0)
    basic, _, _ = oracle.bm3d_pass1(noisy[0], [25.0], oracle.Pass(lambda3d=1e9))
    assert np.abs(basic).max() == 0.0


def test_wiener_with_vanishing_sigma_returns_noisy(oracle):
    _, noisy = synth.make_batch([13], 40, 40, 25.0)
    y = noisy[0].astype(np.float64)
    out, _, _ = oracle.bm3d_pass2(y, y, [1e-4], oracle.Pass(n2=32, tau=400.0))
    np.testing.assert_allclose(out, y, atol=1e-5)


@pytest.mark.parametrize("c,C,sigma", [(100.0, 1, 25.0), (0.0, 1, 25.0), (60.0, 3, 15.0), (150.0, 1, 50.0)])
def test_constant_image_closed_form(oracle, c, C, sigma):
    """A constant image c is a fixed point of the hard-threshold pass (only the
    DC coefficient 8 c sqrt(n) survives).  In the Wiener pass every candidate
    matches (d = 0), so every group has n = 32 equal patches and only the DC
    coefficient B = 8 c sqrt(32) is nonzero: the output is c B^2/(B^2 + sigma^2)."""
    img = np.full((C, 36, 41), c)
    basic, final = oracle.bm3d(img, sigma)
    np.testing.assert_allclose(basic, c, atol=1e-9)
    sy = oracle.channel_sigmas(sigma, C)[0]
    B2 = 64.0 * 32.0 * c * c
    gain = B2 / (B2 + sy * sy)
    np.testing.assert_allclose(final, c * gain, atol=1e-9)


def test_two_patch_weighting_closed_form(oracle):
    """8x9 image, two references (x = 0 and x = 1), tau below their distance so
    each group holds one patch.  Each estimate is the hard-thresholded 2D DCT of
    its patch (scipy), the group weight is 1/(sigma^2 N_har) and each
    contribution is windowed by kaiser(8, 2) (numpy)."""
    rng = np.random.default_rng(0)
    img = 100.0 + rng.normal(0, 30, (8, 9))
    sigma, lam = 10.0, 2.7
    thr = lam * sigma
    est, wts = [], []
    for x0 in (0, 1):
        D = scipy.fft.dctn(img[:, x0:x0 + 8], norm="ortho")
        keep = np.abs(D) > thr
        est.append(scipy.fft.idctn(D * keep, norm="ortho"))
        wts.append(1.0 / (sigma ** 2 * keep.sum()))
    k = np.kaiser(8, 2.0)
    K = np.outer(k, k)
    num = np.zeros((8, 9))
    den = np.zeros((8, 9))
    for x0, e, w in zip((0, 1), est, wts):
        num[:, x0:x0 + 8] += w * K * e
        den[:, x0:x0 + 8] += w * K
    expect = num / den
    d01 = ((img[:, 0:8] - img[:, 1:9]) ** 2).mean()
    basic, _, _ = oracle.bm3d_pass1(img[None], [sigma], oracle.Pass(tau=0.5 * d01, lambda3d=lam))
    np.testing.assert_allclose(basic[0], expect, atol=1e-10)


def test_two_patch_wiener_closed_form(oracle):
    """Same geometry for the Wiener pass: gains B^2/(B^2+sigma^2) on the 2D DCT
    of the basic patch, applied to the noisy patch, weight 1/(sigma^2 sum w^2)."""
    rng = np.random.default_rng(1)
    basic = 100.0 + rng.normal(0, 30, (8, 9))
    noisy = basic + rng.normal(0, 10, (8, 9))
    sigma = 10.0
    k = np.kaiser(8, 2.0)
    K = np.outer(k, k)
    num = np.zeros((8, 9))
    den = np.zeros((8, 9))
    for x0 in (0, 1):
        B = scipy.fft.dctn(basic[:, x0:x0 + 8], norm="ortho")
        Y = scipy.fft.dctn(noisy[:, x0:x0 + 8], norm="ortho")
        om = B ** 2 / (B ** 2 + sigma ** 2)
        e = scipy.fft.idctn(om * Y, norm="ortho")
        w = 1.0 / (sigma ** 2 * (om ** 2).sum())
        num[:, x0:x0 + 8] += w * K * e
        den[:, x0:x0 + 8] += w * K
    d01 = ((basic[:, 0:8] - basic[:, 1:9]) ** 2).mean()
    out, _, _ = oracle.bm3d_pass2(noisy[None], basic[None], [sigma], oracle.Pass(n2=32, tau=0.5 * d01))
    np.testing.assert_allclose(out[0], num / den, atol=1e-10)


def test_two_identical_patches_group_of_two(oracle):
    """8x9 image whose two patches are equal: one group of n = 2 per reference;
    identical patches put the whole group in Hadamard row 0, so the estimate of
    each is the 2D hard threshold at lambda sigma / sqrt(2) of the patch."""
    rng = np.random.default_rng(2)
    img = np.tile(rng.normal(100, 30, (8, 1)), (1, 9))  # constant along x: both patches equal
    sigma, lam = 10.0, 2.7
    D = scipy.fft.dctn(img[:, 0:8], norm="ortho")
    keep = np.sqrt(2.0) * np.abs(D) > lam * sigma
    e = scipy.fft.idctn(D * keep, norm="ortho")
    basic, _, _ = oracle.bm3d_pass1(img[None], [sigma], oracle.Pass(lambda3d=lam))
    np.testing.assert_allclose(basic[0], np.concatenate([e, e[:, :1]], axis=1), atol=1e-10)


def test_colour_transform_round_trip_and_sigmas(oracle):
    x = np.random.default_rng(4).uniform(0, 255, (3, 5, 6))
    np.testing.assert_allclose(oracle.ycc_to_rgb(oracle.rgb_to_ycc(x)), x, atol=1e-10)
    grey = np.full((3, 2, 2), 90.0)
    ycc = oracle.rgb_to_ycc(grey)
    np.testing.assert_allclose(ycc[0], 90.0, atol=1e-12)
    np.testing.assert_allclose(ycc[1:], 0.0, atol=1e-12)
    n = np.random.default_rng(5).normal(0, 25.0, (3, 400, 500))
    emp = oracle.rgb_to_ycc(n).reshape(3, -1).std(axis=1)
    np.testing.assert_allclose(emp, oracle.channel_sigmas(25.0, 3), rtol=0.01)
    np.testing.assert_allclose(oracle.channel_sigmas(25.0, 3), [16.715, 15.578, 16.430], atol=2e-3)


def test_bm3d_denoises_synthetic_scene(oracle):
    clean, noisy = synth.make_batch([0], 96, 96, 25.0)
    basic, final = oracle.bm3d(noisy[0], 25.0)
    p0 = oracle.psnr(noisy[0], clean[0])
    p1 = oracle.psnr(basic, clean[0])
    p2 = oracle.psnr(final, clean[0])
    assert p1 > p0 + 6.0 and p2 > p1


def test_psnr_closed_form(oracle):
    clean = np.full((2, 10, 10), 100.0)
    assert abs(oracle.psnr(clean + 5.0, clean) - 20 * np.log10(255.0 / 5.0)) < 1e-12
    assert oracle.psnr(clean, clean) == float("inf")
    assert abs(oracle.psnr(np.full((1, 4, 4), 300.0), np.full((1, 4, 4), 250.0)) - 20 * np.log10(255.0 / 5)) < 1e-12


# ---- larger patches (the high-noise profile: 12 x 12 step 4, 11 x 11 step 6) ----------

HARD12 = dict(patch=12, step=4, n2=16, tau=5000.0)
WIENER11 = dict(patch=11, step=6, n2=32, tau=3500.0)


@pytest.mark.parametrize("C", [1, 3])
def test_lambda_zero_is_identity_12x12(oracle, C):
    _, noisy = synth.make_batch([14], 41, 37, 50.0, C=C)
    x = noisy[0].astype(np.float64)
    basic, _, _ = oracle.bm3d_pass1(x, [50.0] * C, oracle.Pass(lambda3d=0.0, **HARD12))
    np.testing.assert_allclose(basic, x, atol=1e-9)


@pytest.mark.parametrize("c,sigma", [(100.0, 50.0), (30.0, 60.0)])
def test_constant_image_closed_form_larger_patches(oracle, c, sigma):
    """As the 8 x 8 case: the 12 x 12 hard pass keeps only the DC coefficient
    12 c sqrt(n) (a fixed point); in the 11 x 11 Wiener pass every group has
    32 equal patches and the DC coefficient B = 11 c sqrt(32)."""
    img = np.full((1, 35, 40), c)
    basic, final = oracle.bm3d(img, sigma, hard=oracle.Pass(**HARD12), wiener=oracle.Pass(**WIENER11))
    np.testing.assert_allclose(basic, c, atol=1e-9)
    B2 = 121.0 * 32.0 * c * c
    np.testing.assert_allclose(final, c * B2 / (B2 + sigma * sigma), atol=1e-9)


def test_two_patch_weighting_closed_form_12x12(oracle):
    """12 x 13 image, references x = 0 and x = 1 (step 4 puts the second at
    W - 12 = 1), one patch per group: scipy's 12-point DCT, weight
    1/(sigma^2 N_har) and the kaiser(12, 2) window (numpy)."""
    rng = np.random.default_rng(20)
    img = 100.0 + rng.normal(0, 30, (12, 13))
    sigma, lam = 10.0, 2.7
    k = np.kaiser(12, 2.0)
    K = np.outer(k, k)
    num = np.zeros((12, 13))
    den = np.zeros((12, 13))
    for x0 in (0, 1):
        D = scipy.fft.dctn(img[:, x0:x0 + 12], norm="ortho")
        keep = np.abs(D) > lam * sigma
        e = scipy.fft.idctn(D * keep, norm="ortho")
        w = 1.0 / (sigma ** 2 * keep.sum())
        num[:, x0:x0 + 12] += w * K * e
        den[:, x0:x0 + 12] += w * K
    d01 = ((img[:, 0:12] - img[:, 1:13]) ** 2).mean()
    p = oracle.Pass(patch=12, step=4, tau=0.5 * d01, lambda3d=lam)
    basic, _, _ = oracle.bm3d_pass1(img[None], [sigma], p)
    np.testing.assert_allclose(basic[0], num / den, atol=1e-10)


def test_two_patch_wiener_closed_form_11x11(oracle):
    rng = np.random.default_rng(21)
    basic = 100.0 + rng.normal(0, 30, (11, 12))
    noisy = basic + rng.normal(0, 10, (11, 12))
    sigma = 10.0
    k = np.kaiser(11, 2.0)
    K = np.outer(k, k)
    num = np.zeros((11, 12))
    den = np.zeros((11, 12))
    for x0 in (0, 1):
        B = scipy.fft.dctn(basic[:, x0:x0 + 11], norm="ortho")
        Y = scipy.fft.dctn(noisy[:, x0:x0 + 11], norm="ortho")
        om = B ** 2 / (B ** 2 + sigma ** 2)
        e = scipy.fft.idctn(om * Y, norm="ortho")
        w = 1.0 / (sigma ** 2 * (om ** 2).sum())
        num[:, x0:x0 + 11] += w * K * e
        den[:, x0:x0 + 11] += w * K
    d01 = ((basic[:, 0:11] - basic[:, 1:12]) ** 2).mean()
    p = oracle.Pass(patch=11, step=6, n2=32, tau=0.5 * d01)
    out, _, _ = oracle.bm3d_pass2(noisy[None], basic[None], [sigma], p)
    np.testing.assert_allclose(out[0], num / den, atol=1e-10)


def test_high_noise_profile_denoises_synthetic_scene(oracle):
    clean, noisy = synth.make_batch([1], 80, 80, 50.0)
    basic, final = oracle.bm3d(noisy[0], 50.0, hard=oracle.Pass(lambda2d=2.0, **HARD12),
                               wiener=oracle.Pass(**WIENER11))
    p0 = oracle.psnr(noisy[0], clean[0])
    assert oracle.psnr(basic, clean[0]) > p0 + 6.0 and oracle.psnr(final, clean[0]) > p0 + 6.0

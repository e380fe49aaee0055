"""NL-means and residual-CNN parity of the CUDA path against the FP64 oracle.

NL-means has no discrete decision, so every pixel must agree within 1e-3
(0..255 scale).  CNN layers in FP32 agree with the oracle to 1e-4 relative
to the output scale; the full FP32 network output within 1e-3."""
import numpy as np
import pytest

from gpu_util import dev, host, need_gpu
from paper_2403_03488_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def api():
    from paper_2403_03488_gb300 import api as A
    return A


@pytest.mark.parametrize("C,H,W,sigmas", [(1, 70, 90, (15.0, 50.0)), (3, 41, 37, (25.0,)), (1, 5, 6, (25.0,)),
                                          (1, 8, 130, (25.0,))])
def test_nlm_parity(oracle, C, H, W, sigmas):
    A = api()
    B = len(sigmas)
    _, noisy = synth.make_batch(range(60, 60 + B), H, W, list(sigmas), C=C)
    out = host(A.denoise_nlm(dev(noisy), list(sigmas)))
    for b in range(B):
        ref = oracle.nlm_image(noisy[b], sigmas[b])
        err = np.abs(out[b] - ref).max()
        assert err <= TOL, (b, err)


@pytest.mark.parametrize("C,patch,search", [(1, 5, 11), (1, 9, 25), (3, 3, 15), (1, 7, 19), (1, 7, 41), (1, 5, 1),
                                             (1, 3, 21), (1, 11, 21)])
def test_nlm_parity_other_patch_and_search(oracle, C, patch, search):
    """Non-default neighbourhood and window sizes (the kernels' halos, tile
    loops and masked offset lanes follow the parameters; odd and even search
    radii, the largest window, a window of one offset)."""
    A = api()
    _, noisy = synth.make_batch([66], 45, 71, 25.0, C=C)
    p = A.default_nlm_params()
    p.patch, p.search = patch, search
    out = host(A.denoise_nlm(dev(noisy), [25.0], p))
    ref = oracle.nlm_image(noisy[0], 25.0, patch, search)
    assert np.abs(out[0] - ref).max() <= TOL


def test_nlm_full_size_sampled(oracle):
    """8 x 512 x 512 (the plain-method batch): 200 sampled pixels against the
    oracle run on crops holding each pixel's search window and patches."""
    A = api()
    _, noisy = synth.make_batch(range(8), 512, 512, 25.0)
    out = host(A.denoise_nlm(dev(noisy), 25.0))
    rng = np.random.default_rng(2)
    for _ in range(200):
        b, y, x = int(rng.integers(0, 8)), int(rng.integers(0, 512)), int(rng.integers(0, 512))
        if rng.random() < 0.2:
            y = int(rng.choice([0, 1, 2, 510, 511]))
        y0, y1, x0, x1 = max(0, y - 13), min(512, y + 14), max(0, x - 13), min(512, x + 14)
        ref = oracle.nlm(noisy[b, 0, y0:y1, x0:x1], 25.0)[y - y0, x - x0]
        assert abs(out[b, 0, y, x] - ref) <= TOL


@pytest.mark.parametrize("N,Cin,Cout,H,W", [(2, 2, 32, 19, 23), (1, 32, 32, 33, 17), (3, 32, 1, 16, 16),
                                            (1, 5, 7, 1, 9)])
def test_conv3x3_fwd_bwd_parity(oracle, N, Cin, Cout, H, W):
    A = api()
    rng = np.random.default_rng(N * 7 + Cin)
    x = rng.normal(0, 1, (N, Cin, H, W)).astype(np.float32)
    w = (rng.normal(0, 1, (Cout, 3, 3, Cin)) * np.sqrt(2.0 / (9 * Cin))).astype(np.float32)
    b = rng.normal(0, 0.1, Cout).astype(np.float32)
    dy = rng.normal(0, 1, (N, Cout, H, W)).astype(np.float32)
    y = host(A.conv3x3_fwd(dev(x), dev(w), dev(b), relu=False))
    yr = oracle.conv3x3(x, w, b)
    assert np.abs(y - yr).max() <= 1e-4 * max(1.0, np.abs(yr).max())
    yrelu = host(A.conv3x3_fwd(dev(x), dev(w), dev(b), relu=True))
    assert np.abs(yrelu - np.maximum(yr, 0)).max() <= 1e-4 * max(1.0, np.abs(yr).max())
    dxr, dwr, dbr = oracle.conv3x3_bwd(x, dy, w)
    dx = host(A.conv3x3_bwd_data(dev(dy), dev(w)))
    assert np.abs(dx - dxr).max() <= 1e-4 * max(1.0, np.abs(dxr).max())
    mask = (rng.random(x.shape) > 0.5).astype(np.float32)
    dxm = host(A.conv3x3_bwd_data(dev(dy), dev(w), dev(mask)))
    assert np.abs(dxm - dxr * (mask > 0)).max() <= 1e-4 * max(1.0, np.abs(dxr).max())
    dw, db = A.conv3x3_bwd_weight(dev(x), dev(dy))
    dw, db = host(dw), host(db)
    assert np.abs(dw - dwr).max() <= 1e-4 * max(1.0, np.abs(dwr).max())
    assert np.abs(db - dbr).max() <= 1e-4 * max(1.0, np.abs(dbr).max())


def _flat(params):
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in params]).astype(np.float32)


@pytest.mark.parametrize("N,H,W", [(2, 37, 29), (1, 64, 64)])
def test_cnn_forward_fp32_parity(oracle, N, H, W):
    A = api()
    rng = np.random.default_rng(3)
    params = synth.he_normal_weights(7, layers=10, width=32)
    params = [(w, rng.normal(0, 0.05, b.shape).astype(np.float32)) for w, b in params]
    clean = rng.uniform(0, 255, (N, H, W)).astype(np.float32)
    noisy = (clean + rng.normal(0, 25, clean.shape)).astype(np.float32)
    pre = (clean + rng.normal(0, 5, clean.shape)).astype(np.float32)
    out = host(A.cnn_forward(dev(noisy), dev(pre), dev(_flat(params)), 10, 32))
    ref = oracle.cnn_forward(noisy, pre, params)
    assert np.abs(out - ref).max() <= TOL


def test_l1_grad_and_adam(oracle):
    A = api()
    import torch
    rng = np.random.default_rng(4)
    r = rng.normal(0, 0.1, (2, 9, 11)).astype(np.float32)
    pre = rng.uniform(0, 255, r.shape).astype(np.float32)
    clean = rng.uniform(0, 255, r.shape).astype(np.float32)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    dr = host(A.l1_residual_grad(dev(r), dev(pre), dev(clean), loss))
    out = pre.astype(np.float64) + 255.0 * r
    np.testing.assert_allclose(dr, 255.0 * np.sign(out - clean) / r.size, rtol=1e-6)
    assert abs(host(loss)[0] / r.size - oracle.l1_loss(out, clean)) < 1e-4
    p = rng.normal(0, 1, 50).astype(np.float32)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    pt, mt, vt = dev(p.copy()), dev(m.copy()), dev(v.copy())
    pr, mr, vr = p.astype(np.float64), m.astype(np.float64), v.astype(np.float64)
    for t in range(1, 4):
        g = rng.normal(0, 1, 50).astype(np.float32)
        A.adam_step(pt, dev(g), mt, vt, t)
        pr, mr, vr = oracle.adam_step(pr, g.astype(np.float64), mr, vr, t)
    np.testing.assert_allclose(host(pt), pr, atol=1e-6)


def _bf16(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16).float().numpy()


@pytest.mark.parametrize("N,H,W,relu,C", [(2, 5, 200, True, 32), (1, 37, 128, False, 32), (1, 3, 1, True, 32),
                                          (3, 17, 131, True, 32), (1, 37, 131, True, 64), (2, 5, 9, False, 64)])
def test_conv3x3_tc_bf16_parity(oracle, N, H, W, relu, C):
    """tcgen05 hidden layer vs the FP64 oracle on the same BF16-rounded inputs and
    weights: only FP32 accumulation and the final BF16 rounding differ
    (<= 2 BF16 ulps of the output plus 1e-3 of its scale)."""
    import torch
    A = api()
    rng = np.random.default_rng(N * 100 + W + C)
    x = _bf16(np.maximum(rng.normal(0, 1, (N, C, H, W)), 0))
    w = _bf16(rng.normal(0, 1, (C, 3, 3, C)) * np.sqrt(2.0 / (9 * C)))
    b = rng.normal(0, 0.1, C).astype(np.float32)
    ref = oracle.conv3x3(x, w, b)
    if relu:
        ref = np.maximum(ref, 0)
    xt = torch.from_numpy(x).permute(0, 2, 3, 1).contiguous().to(torch.bfloat16).cuda()
    y = A.conv3x3_tc_fwd(xt, dev(w), dev(b), relu=relu)
    got = host(y.float().permute(0, 3, 1, 2))
    scale = np.abs(ref).max()
    assert np.all(np.abs(got - ref) <= 2 ** -7 * np.abs(ref) + 1e-3 * scale)
    assert A.device_error() == 0


def test_conv3x3_tc_bf16_more_work_items_than_ctas():
    """Persistent tcgen05 conv with more (image, strip, 32-row chunk) items than
    resident CTAs (500 items: ragged last strip and chunk), against an FP64
    convolution of the same BF16-rounded operands (FP64 on the GPU: cuDNN's
    FP32 convolutions may run in TF32, narrower than the kernel's FP32
    accumulation)."""
    import torch
    A = api()
    N, H, W = 10, 300, 520
    g = torch.Generator(device="cuda").manual_seed(5)
    x = torch.relu(torch.randn(N, H, W, 32, device="cuda", generator=g)).to(torch.bfloat16)
    w = (torch.randn(32, 3, 3, 32, device="cuda", generator=g) * (2.0 / 288) ** 0.5).to(torch.bfloat16).float()
    b = torch.randn(32, device="cuda", generator=g) * 0.1
    y = A.conv3x3_tc_fwd(x, w.contiguous(), b, relu=True)
    ref = torch.relu(torch.nn.functional.conv2d(x.double().permute(0, 3, 1, 2), w.double().permute(0, 3, 1, 2),
                                                b.double(), padding=1))
    got = y.double().permute(0, 3, 1, 2)
    scale = ref.abs().max()
    assert bool(((got - ref).abs() <= 2 ** -7 * ref.abs() + 1e-3 * scale).all())
    assert A.device_error() == 0


def test_conv3x3_tc64_bf16_more_work_items_than_ctas():
    """64-channel tcgen05 layer (one CTA per SM) with 5 x 3 x 10 = 150 work
    items over 152 CTAs plus ragged strips/chunks, against an FP64 convolution
    on the GPU."""
    import torch
    A = api()
    N, H, W = 5, 300, 300
    g = torch.Generator(device="cuda").manual_seed(6)
    x = torch.relu(torch.randn(N, H, W, 64, device="cuda", generator=g)).to(torch.bfloat16)
    w = (torch.randn(64, 3, 3, 64, device="cuda", generator=g) * (2.0 / 576) ** 0.5).to(torch.bfloat16).float()
    b = torch.randn(64, device="cuda", generator=g) * 0.1
    y = A.conv3x3_tc_fwd(x, w.contiguous(), b, relu=False)
    ref = torch.nn.functional.conv2d(x.double().permute(0, 3, 1, 2), w.double().permute(0, 3, 1, 2), b.double(),
                                     padding=1)
    got = y.double().permute(0, 3, 1, 2)
    scale = ref.abs().max()
    assert bool(((got - ref).abs() <= 2 ** -7 * ref.abs() + 1e-3 * scale).all())
    assert A.device_error() == 0


def _colour_case(seed, H, W):
    rng = np.random.default_rng(seed)
    clean = rng.uniform(0, 255, (2, 3, H, W)).astype(np.float32)
    noisy = (clean + rng.normal(0, 25, clean.shape)).astype(np.float32)
    pre = (clean + rng.normal(0, 5, clean.shape)).astype(np.float32)
    return noisy, pre


def test_cnn_forward_fp32_colour_native_k16_matches_oracle(oracle):
    """Colour-native network (6 -> 32 -> ... -> 3, K = 16) on the FP32 path."""
    A = api()
    rng = np.random.default_rng(11)
    params = synth.he_normal_weights(12, layers=16, width=32, cin=6, cout=3)
    params = [(w * 0.6, rng.normal(0, 0.02, b.shape).astype(np.float32)) for w, b in params]
    noisy, pre = _colour_case(12, 23, 37)
    out = host(A.cnn_forward(dev(noisy), dev(pre), dev(_flat(params)), 16, 32, precision=A.DN_FP32))
    ref = oracle.cnn_forward(noisy, pre, params)
    assert out.shape == ref.shape == (2, 3, 23, 37)
    assert np.abs(out - ref).max() <= 1e-3 * max(1.0, np.abs(ref - pre).max())


@pytest.mark.parametrize("layers,width,colour", [(10, 32, True), (10, 64, False), (16, 64, True)])
def test_cnn_forward_bf16_wider_and_colour_close_to_oracle(oracle, layers, width, colour):
    """tcgen05 path for the shapes beyond 10 x 32 grey: 64 channels (one CTA per
    SM), colour-native input/output planes, K = 16."""
    A = api()
    rng = np.random.default_rng(layers * width)
    cc = 3 if colour else 1
    params = synth.he_normal_weights(5, layers=layers, width=width, cin=2 * cc, cout=cc)
    params = [(w * 0.5, rng.normal(0, 0.02, b.shape).astype(np.float32)) for w, b in params]
    noisy, pre = _colour_case(layers + width, 21, 140)
    if not colour:
        noisy, pre = noisy[:, 0], pre[:, 0]
    out = host(A.cnn_forward(dev(noisy), dev(pre), dev(_flat(params)), layers, width, precision=A.DN_BF16))
    ref = oracle.cnn_forward(noisy, pre, params)
    r = np.abs(ref - pre).max()
    assert np.abs(out - ref).max() <= 0.03 * r + 1e-2
    assert A.device_error() == 0


def test_hybrid_with_colour_native_network():
    """denoise_hybrid with a colour-native network: RGB only (grey input is
    refused), BF16 tcgen05 close to the FP32 path."""
    import torch
    from paper_2403_03488_gb300 import _lib as L
    A = api()
    rng = np.random.default_rng(21)
    params = synth.he_normal_weights(21, layers=10, width=32, cin=6, cout=3)
    params = [(w * 0.5, rng.normal(0, 0.02, b.shape).astype(np.float32)) for w, b in params]
    wts = dev(_flat(params))
    _, noisy = synth.make_batch([61, 62], 48, 56, [25.0, 15.0], C=3)
    x = dev(noisy)
    f32 = host(A.denoise_hybrid(x, [25.0, 15.0], wts, cnn_precision=A.DN_FP32, cnn_channels=3))
    b16 = host(A.denoise_hybrid(x, [25.0, 15.0], wts, cnn_precision=A.DN_BF16, cnn_channels=3))
    pre = host(A.denoise_bm3d(x, [25.0, 15.0]))
    assert np.isfinite(b16).all()
    assert np.abs(b16 - f32).max() <= 0.03 * np.abs(f32 - pre).max() + 1e-2
    with pytest.raises(L.DenoiseError):
        A.denoise_hybrid(x[:, :1].contiguous(), [25.0, 15.0], wts, cnn_channels=3)


def test_cnn_forward_bf16_close_to_oracle(oracle):
    A = api()
    rng = np.random.default_rng(8)
    params = synth.he_normal_weights(3, layers=10, width=32)
    params = [(w * 0.5, rng.normal(0, 0.02, b.shape).astype(np.float32)) for w, b in params]
    clean = rng.uniform(0, 255, (2, 45, 140)).astype(np.float32)
    noisy = (clean + rng.normal(0, 25, clean.shape)).astype(np.float32)
    pre = (clean + rng.normal(0, 5, clean.shape)).astype(np.float32)
    out = host(A.cnn_forward(dev(noisy), dev(pre), dev(_flat(params)), 10, 32, precision=A.DN_BF16))
    ref = oracle.cnn_forward(noisy, pre, params)
    r = np.abs(ref - pre).max()
    assert np.abs(out - ref).max() <= 0.03 * r + 1e-2
    assert A.device_error() == 0


@pytest.mark.parametrize("N,H,W", [(2, 70, 300), (1, 33, 126), (3, 64, 127), (1, 1, 9), (16, 256, 256)])
def test_conv3x3_tc_pair_equals_two_layers(N, H, W):
    """Two hidden layers fused in one pass (the intermediate rows kept in
    shared memory, strips of 126 output pixels) give bit for bit the result of
    two single-layer launches: same BF16 rounding of the intermediate, same
    MMA order.  Ragged strips and items, strip-wide and one-row images."""
    import torch
    A = api()
    g = torch.Generator(device="cuda").manual_seed(N * 7 + H + W)
    x = torch.relu(torch.randn(N, H, W, 32, device="cuda", generator=g)).to(torch.bfloat16)
    wa = torch.randn(32, 3, 3, 32, device="cuda", generator=g) * (2.0 / 288) ** 0.5
    wb = torch.randn(32, 3, 3, 32, device="cuda", generator=g) * (2.0 / 288) ** 0.5
    ba = torch.randn(32, device="cuda", generator=g) * 0.1
    bb = torch.randn(32, device="cuda", generator=g) * 0.1
    two = A.conv3x3_tc_fwd(A.conv3x3_tc_fwd(x, wa, ba, relu=True), wb, bb, relu=True)
    fused = A.conv3x3_tc_pair_fwd(x, wa, ba, wb, bb)
    assert torch.equal(two.view(torch.int16), fused.view(torch.int16))
    assert A.device_error() == 0

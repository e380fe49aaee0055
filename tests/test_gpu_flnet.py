"""The flexible lightweight network (Sec. III) on the GPU against the FP64
oracle: every layer kernel forward and backward (odd sizes, channel counts
that are not multiples of the kernels' channel blocks, stride 2), the whole
network's output and gradients, one L1 + Adam training step, and a short
training run that lowers the loss."""
import numpy as np
import pytest

from gpu_util import dev, host, need_gpu

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def A():
    from paper_2403_03488_gb300 import api
    return api


def ref_grads(fn, *arrays):
    ts = [torch.as_tensor(np.asarray(a, np.float64)).requires_grad_(True) for a in arrays]
    return fn(*ts), ts


def close(a, b, rel=1e-5):
    b = np.asarray(b, np.float64)
    assert np.abs(np.asarray(a, np.float64) - b).max() <= rel * max(1.0, np.abs(b).max()), (
        np.abs(np.asarray(a, np.float64) - b).max(), np.abs(b).max())


@pytest.mark.parametrize("stride,relu,shape", [(1, False, (2, 5, 13, 18)), (2, False, (2, 5, 13, 18)),
                                               (1, True, (2, 5, 13, 18)), (2, True, (2, 5, 13, 18)),
                                               (1, True, (2, 3, 70, 301)), (2, False, (3, 3, 71, 600)),
                                               (1, True, (2, 3, 37, 520)), (2, True, (2, 5, 13, 16)),
                                               (1, False, (1, 4, 21, 1032))])
def test_depthwise_forward_and_backward(oracle, stride, relu, shape):
    """Small planes, and planes with several row bands and column chunks
    (ragged in both) for the banded forward kernels; widths that are multiples
    of 4 (stride 1) or 8 (stride 2) take the float4 form."""
    _, F = oracle._fl_torch()
    rng = np.random.default_rng(stride)
    C = shape[1]
    x = rng.standard_normal(shape).astype(np.float32)
    w = rng.standard_normal((C, 3, 3)).astype(np.float32)
    b = rng.standard_normal(C).astype(np.float32)
    y = host(A().dw3x3_fwd(dev(x), dev(w), dev(b), stride=stride, relu=relu))
    yr, (tx, tw, tb) = ref_grads(lambda X, Wt, B: F.conv2d(X, Wt.reshape(C, 1, 3, 3), B, stride=stride, padding=1,
                                                           groups=C), x, w, b)
    close(y, (yr.clamp(min=0) if relu else yr).detach().numpy())
    g = rng.standard_normal(yr.shape).astype(np.float32)
    yr.backward(torch.as_tensor(g, dtype=torch.float64))
    dx, dw, db = A().dw3x3_bwd(dev(x), dev(g), dev(w), stride=stride)
    close(host(dx), tx.grad.numpy())
    close(host(dw), tw.grad.numpy(), 1e-4)
    close(host(db), tb.grad.numpy(), 1e-4)


@pytest.mark.parametrize("relu,shape,cout", [(False, (2, 20, 7, 9), 37), (True, (2, 20, 7, 9), 37),
                                             (True, (3, 21, 37, 41), 18), (False, (1, 3, 64, 33), 48),
                                             (True, (2, 21, 16, 20), 18)])
def test_pointwise_forward_and_backward(oracle, relu, shape, cout):
    """Channel counts off the 4-channel load groups and the 16-channel blocks,
    pixel counts over several 512-pixel tiles with a ragged tail; the last two
    shapes (pixels per image a multiple of 4) take the float4 kernel."""
    _, F = oracle._fl_torch()
    rng = np.random.default_rng(7)
    cin = shape[1]
    x = rng.standard_normal(shape).astype(np.float32)
    w = rng.standard_normal((cout, cin)).astype(np.float32)
    b = rng.standard_normal(cout).astype(np.float32)
    y = host(A().pw_fwd(dev(x), dev(w), dev(b), relu=relu))
    yr, (tx, tw, tb) = ref_grads(lambda X, Wt, B: F.conv2d(X, Wt.reshape(cout, cin, 1, 1), B), x, w, b)
    close(y, (yr.clamp(min=0) if relu else yr).detach().numpy())
    g = rng.standard_normal(yr.shape).astype(np.float32)
    yr.backward(torch.as_tensor(g, dtype=torch.float64))
    close(host(A().pw_fwd(dev(g), dev(w), None, transposed=True)), tx.grad.numpy())
    dw, db = A().pw_bwd_weight(dev(x), dev(g))
    close(host(dw), tw.grad.numpy(), 1e-4)
    close(host(db), tb.grad.numpy(), 1e-4)


@pytest.mark.parametrize("shape", [(2, 13, 5, 6), (2, 13, 5, 8), (1, 7, 9, 36)])
def test_transposed_convolution_forward_and_backward(oracle, shape):
    """Odd channel counts; widths that are multiples of 4 take the float4 kernel."""
    _, F = oracle._fl_torch()
    rng = np.random.default_rng(9)
    n, cin, h, wd = shape
    x = rng.standard_normal(shape).astype(np.float32)
    w = rng.standard_normal((cin, 11, 2, 2)).astype(np.float32)
    b = rng.standard_normal(11).astype(np.float32)
    skip = rng.standard_normal((n, 11, 2 * h, 2 * wd)).astype(np.float32)
    y = host(A().deconv2x2_fwd(dev(x), dev(w), dev(b), dev(skip)))
    yr, (tx, tw, tb) = ref_grads(lambda X, Wt, B: F.conv_transpose2d(X, Wt, B, stride=2), x, w, b)
    close(y, yr.detach().numpy() + skip)
    g = rng.standard_normal(yr.shape).astype(np.float32)
    yr.backward(torch.as_tensor(g, dtype=torch.float64))
    dx, dw, db = A().deconv2x2_bwd(dev(x), dev(g), dev(w))
    close(host(dx), tx.grad.numpy())
    close(host(dw), tw.grad.numpy(), 1e-4)
    close(host(db), tb.grad.numpy(), 1e-4)


def _batch(seed, n, h, w):
    from paper_2403_03488_gb300 import synth
    sig = [15.0, 50.0, 25.0, 35.0][:n]
    clean, noisy = synth.make_batch(range(seed, seed + n), h, w, sig)
    rng = np.random.default_rng(seed)
    pre = (clean[:, 0] + rng.normal(0, 4, clean[:, 0].shape)).astype(np.float32)  # a prefilter-like input
    return clean[:, 0], noisy[:, 0], pre, sig


@pytest.mark.parametrize("widths,h,w", [((8, 12, 16, 20, 24), 32, 48), (None, 32, 32)])
def test_network_forward_and_gradients_match_oracle(oracle, widths, h, w):
    from paper_2403_03488_gb300.flnet import FLNet, WIDTHS
    widths = widths or WIDTHS
    clean, noisy, pre, sig = _batch(600, 2, h, w)
    net = FLNet(widths, seed=3).cuda()
    with torch.no_grad():  # nonzero biases so that every bias path is exercised
        net.flat.add_(0.01 * torch.sin(torch.arange(net.flat.numel(), device="cuda", dtype=torch.float32)))
    prm = net.numpy_params()
    out = host(net(dev(noisy), dev(pre), sig))
    ref = oracle.fl_forward(noisy, pre, sig, prm)
    # an untrained network's outputs reach ~1e4 grey levels: FP32 relative error
    assert np.abs(out - ref).max() <= 2e-5 * max(255.0, np.abs(ref).max()), (np.abs(out - ref).max(), np.abs(ref).max())
    # gradients of the L1 loss through the library's backward kernels
    r = net.residual(dev(noisy), dev(pre), sig).contiguous()
    dr = A().l1_residual_grad(r, dev(pre), dev(clean))
    r.backward(dr)
    gflat = net.flat.grad.detach()
    _, grads = oracle.fl_backward(noisy, pre, clean, sig, prm)
    for o, s, gref in zip(net.offsets, net.shapes, grads):
        g = host(gflat[o:o + int(np.prod(s))]).reshape(s)
        assert np.abs(g - gref).max() <= 2e-4 * max(1e-3, np.abs(gref).max()), (s, np.abs(g - gref).max(),
                                                                               np.abs(gref).max())


def test_training_step_matches_oracle_adam(oracle):
    from paper_2403_03488_gb300.flnet import FLNet
    widths = (8, 12, 16, 20, 24)
    clean, noisy, pre, sig = _batch(700, 2, 32, 32)
    net = FLNet(widths, seed=5).cuda()
    before = net.numpy_params()
    loss = net.train_step(dev(noisy), dev(pre), dev(clean), sig, lr=1e-3)
    lref, grads = oracle.fl_backward(noisy, pre, clean, sig, before)
    assert abs(loss - lref) <= 1e-4 * lref
    after = net.numpy_params()
    for p0, p1, g in zip(before, after, grads):
        exp, _, _ = oracle.adam_step(p0.astype(np.float64), g, np.zeros_like(g), np.zeros_like(g), 1)
        # Adam's first step moves every coordinate by ~lr * sign(g): compare where |g| is not tiny
        m = np.abs(g) > 1e-3 * max(1e-6, np.abs(g).max())
        assert np.abs(p1 - exp)[m].max() <= 2e-6 if m.any() else True


def test_short_training_lowers_the_loss():
    from paper_2403_03488_gb300.flnet import FLNet
    clean, noisy, pre, sig = _batch(800, 4, 64, 64)
    net = FLNet((16, 24, 32, 48, 64), seed=1).cuda()
    xs = [dev(a) for a in (noisy, pre, clean)]
    losses = [net.train_step(*xs, sig, lr=2e-3) for _ in range(60)]
    assert np.isfinite(losses).all()
    assert np.mean(losses[-10:]) < 0.8 * np.mean(losses[:5]), (losses[:5], losses[-10:])
    assert A().device_error() == 0


# ---- the tensor-core (BF16 operand) contractions -------------------------------------
# Each output of a pointwise or transposed-convolution layer is a sum of
# products w x with both factors rounded to BF16 (unit roundoff 2^-8) and the
# products accumulated in FP32: |y - exact| <= (2^-7 + 2^-14) sum |w| |x|.

def _bf16_bound(absprod):
    return (2.0 ** -7 + 2.0 ** -14) * absprod + 1e-6


@pytest.mark.parametrize("cin,cout,shape,transposed", [(3, 48, (2, 37, 50), False), (48, 48, (1, 64, 128), False),
                                                       (192, 96, (2, 16, 30), False), (96, 192, (1, 33, 70), True),
                                                       (48, 1, (3, 20, 20), False), (128, 192, (1, 8, 8), False),
                                                       (64, 48, (1, 9, 7), True)])
def test_pointwise_bf16_within_bound(cin, cout, shape, transposed):
    import torch.nn.functional as F
    rng = np.random.default_rng(cin * 7 + cout)
    N, H, W = shape
    x = rng.normal(0, 1, (N, cin, H, W)).astype(np.float32)
    w = (rng.normal(0, 1, (cin, cout) if transposed else (cout, cin)) / np.sqrt(cin)).astype(np.float32)
    b = rng.normal(0, 0.1, cout).astype(np.float32)
    for relu in (False, True):
        y = host(A().pw_fwd(dev(x), dev(w), dev(b), relu=relu, transposed=transposed, precision=A().DN_BF16))
        wm = (w.T if transposed else w).astype(np.float64)
        t = lambda a, ww: F.conv2d(torch.as_tensor(a, dtype=torch.float64), torch.as_tensor(ww)[:, :, None, None])
        ref = t(x, wm).numpy() + b[None, :, None, None]
        bound = _bf16_bound(t(np.abs(x), np.abs(wm)).numpy())
        if relu:
            ref = np.maximum(ref, 0.0)
        assert np.all(np.abs(y - ref) <= bound), np.abs(y - ref).max()
    assert A().device_error() == 0


@pytest.mark.parametrize("cin,cout,shape", [(192, 128, (2, 8, 8)), (64, 48, (1, 33, 40)), (96, 64, (2, 16, 22))])
def test_transposed_convolution_bf16_within_bound(cin, cout, shape):
    import torch.nn.functional as F
    rng = np.random.default_rng(cin + cout)
    N, H, W = shape
    x = rng.normal(0, 1, (N, cin, H, W)).astype(np.float32)
    w = (rng.normal(0, 1, (cin, cout, 2, 2)) / np.sqrt(cin)).astype(np.float32)
    b = rng.normal(0, 0.1, cout).astype(np.float32)
    skip = rng.normal(0, 1, (N, cout, 2 * H, 2 * W)).astype(np.float32)
    y = host(A().deconv2x2_fwd(dev(x), dev(w), dev(b), dev(skip), precision=A().DN_BF16))
    t = lambda a, ww: F.conv_transpose2d(torch.as_tensor(a, dtype=torch.float64), torch.as_tensor(ww, dtype=torch.float64),
                                         stride=2).numpy()
    ref = t(x, w) + b[None, :, None, None] + skip
    assert np.all(np.abs(y - ref) <= _bf16_bound(t(np.abs(x), np.abs(w))))
    assert A().device_error() == 0


def test_network_bf16_close_to_oracle_and_fp32():
    """The trained network with its contractions on the tensor cores against
    the FP64 oracle.  Its ~20 contractions each round activations of up to a
    few hundred times the residual's size to BF16, so the bound is stated on
    the intensity scale, not relative to the (small) residual: every output
    within one grey level of the oracle's, and PSNR within 0.05 dB of the
    oracle's and of the FP32 path's on synthetic scenes."""
    import os
    import oracle
    from paper_2403_03488_gb300 import synth
    from paper_2403_03488_gb300.flnet import FLNet
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    wf = os.path.join(root, "paper_2403_03488_gb300", "weights", "flnet_bm3d.npy")
    flat = torch.from_numpy(np.load(wf).astype(np.float32)) if os.path.exists(wf) else None
    fp32 = (FLNet(flat=flat) if flat is not None else FLNet(seed=0)).cuda()
    bf16 = FLNet(flat=fp32.flat.detach().cpu(), precision=A().DN_BF16).cuda()
    clean, noisy = synth.make_batch([71, 72], 96, 160, 25.0)
    pre = (clean[:, 0] + np.random.default_rng(3).normal(0, 4, clean[:, 0].shape)).astype(np.float32)
    with torch.no_grad():
        o16 = host(bf16(dev(noisy[:, 0]), dev(pre), [25.0, 25.0]))
        o32 = host(fp32(dev(noisy[:, 0]), dev(pre), [25.0, 25.0]))
    ref = oracle.fl_forward(noisy[:, 0], pre, [25.0, 25.0], fp32.numpy_params())
    assert np.abs(o16 - ref).max() <= 1.0, np.abs(o16 - ref).max()
    for k in range(2):
        assert abs(oracle.psnr(o16[k], clean[k, 0]) - oracle.psnr(o32[k], clean[k, 0])) <= 0.05
        assert abs(oracle.psnr(o16[k], clean[k, 0]) - oracle.psnr(ref[k], clean[k, 0])) <= 0.05
    assert A().device_error() == 0

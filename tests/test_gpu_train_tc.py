"""Training of the residual CNN on the tensor cores (BF16 operands, FP32
accumulation and master weights) against the FP64 oracle.

Layer kernels: the weight gradient of a hidden layer (a tcgen05 GEMM over
the pixels) multiplies BF16 values exactly in FP32, so against the oracle's
FP64 sum of the same BF16 inputs it is off only by FP32 accumulation:
|dw - ref| <= 1e-4 sum_px |g| |x| per entry.  The data gradient (tcgen05
transposed convolution, output rounded to BF16) is held to the forward
layer's bound 2^-7 |ref| + 1e-3 max |ref|, and its ReLU mask must zero
exactly the masked entries.

Whole network (dn_cnn_grad): every activation and gradient plane is stored
in BF16 (unit roundoff 2^-8), so each layer's gradient differs from the FP64
oracle's (which the oracle tests pin by central finite differences) by a
few BF16 roundings per layer, propagated through the network: the test
asks for relative Frobenius error <= 5e-2 and cosine >= 0.998 per tensor, and
the loss (from the BF16 forward, whose output error is a few 2^-8 of the
residual) within 5e-3 relative.  Training at batch 64 of 64 x 64 crops must
lower the loss like the FP32 path and take less time per step."""
import time

import numpy as np
import pytest

from gpu_util import dev, host, need_gpu
from paper_2403_03488_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _bf16(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).float().numpy()


@pytest.mark.parametrize("N,H,W", [(3, 37, 150), (2, 64, 64), (1, 9, 260)])
def test_bwd_weight_tc_matches_oracle(oracle, N, H, W):
    import torch
    from paper_2403_03488_gb300 import api
    rng = np.random.default_rng(N * 1000 + H + W)
    x = _bf16(np.maximum(rng.normal(0, 1, (N, 32, H, W)), 0))
    g = _bf16(rng.normal(0, 1, (N, 32, H, W)))
    xt = torch.from_numpy(x).permute(0, 2, 3, 1).contiguous().to(torch.bfloat16).cuda()
    gt = torch.from_numpy(g).permute(0, 2, 3, 1).contiguous().to(torch.bfloat16).cuda()
    dw, db = api.conv3x3_tc_bwd_weight(xt, gt)
    w0 = np.zeros((32, 3, 3, 32))
    _, rdw, rdb = oracle.conv3x3_bwd(x, g, w0)
    _, adw, adb = oracle.conv3x3_bwd(np.abs(x), np.abs(g), w0)
    assert np.all(np.abs(host(dw) - rdw) <= 1e-4 * adw + 1e-6)
    assert np.all(np.abs(host(db) - rdb) <= 1e-4 * adb + 1e-6)
    assert api.device_error() == 0


def test_bwd_data_tc_matches_oracle(oracle):
    import torch
    from paper_2403_03488_gb300 import api
    rng = np.random.default_rng(7)
    N, H, W = 2, 45, 140
    g = _bf16(rng.normal(0, 1, (N, 32, H, W)))
    w = _bf16(rng.normal(0, 0.08, (32, 3, 3, 32)))
    mask = _bf16(np.maximum(rng.normal(0, 1, (N, 32, H, W)), 0))
    gt = torch.from_numpy(g).permute(0, 2, 3, 1).contiguous().to(torch.bfloat16).cuda()
    mt = torch.from_numpy(mask).permute(0, 2, 3, 1).contiguous().to(torch.bfloat16).cuda()
    dx = api.conv3x3_tc_bwd_data(gt, dev(w), mt)
    got = host(dx.float().permute(0, 3, 1, 2))
    rdx, _, _ = oracle.conv3x3_bwd(np.zeros((N, 32, H, W)), g, w)
    ref = rdx * (mask > 0)
    scale = np.abs(ref).max()
    assert np.all(got[mask <= 0] == 0.0)
    assert np.all(np.abs(got - ref) <= 2 ** -7 * np.abs(ref) + 1e-3 * scale)
    assert api.device_error() == 0


def _case(seed, N, H, W):
    rng = np.random.default_rng(seed)
    clean = rng.uniform(0, 255, (N, H, W)).astype(np.float32)
    noisy = (clean + rng.normal(0, 25, clean.shape)).astype(np.float32)
    pre = (clean + rng.normal(0, 6, clean.shape)).astype(np.float32)
    return clean, noisy, pre


def test_cnn_grad_bf16_close_to_oracle(oracle):
    import torch
    from paper_2403_03488_gb300 import api
    from paper_2403_03488_gb300.autograd import ResidualNet
    clean, noisy, pre = _case(4, 4, 40, 48)
    net = ResidualNet(10, 32, seed=4)
    params = net.numpy_params()
    flat = net.flat.detach().cuda()
    grad, loss = api.cnn_grad(dev(noisy), dev(pre), dev(clean), flat)
    ref_loss, grads = oracle.cnn_backward(noisy, pre, clean, params)
    assert abs(float(host(loss)[0]) / clean.size - ref_loss) <= 5e-3 * ref_loss
    mine = ResidualNet(10, 32, flat=torch.from_numpy(host(grad).copy())).numpy_params()
    worst = []
    for (gw, gb), (rw, rb) in zip(mine, grads):
        for a, r in ((gw, rw), (gb, rb)):
            rel = np.linalg.norm(a - r) / max(np.linalg.norm(r), 1e-30)
            cos = float((a * r).sum() / max(np.linalg.norm(a) * np.linalg.norm(r), 1e-30))
            worst.append((rel, cos))
            assert rel <= 5e-2 and cos >= 0.998, (rel, cos)
    print("BF16 network gradient vs FP64 oracle: worst relative error %.3g, worst cosine %.5f" % (
        max(w[0] for w in worst), min(w[1] for w in worst)))
    assert api.device_error() == 0


def test_cnn_grad_bf16_is_reproducible():
    from paper_2403_03488_gb300 import api
    from paper_2403_03488_gb300.autograd import ResidualNet
    clean, noisy, pre = _case(5, 3, 50, 70)
    flat = ResidualNet(10, 32, seed=5).flat.detach().cuda()
    g1, l1 = api.cnn_grad(dev(noisy), dev(pre), dev(clean), flat)
    g2, l2 = api.cnn_grad(dev(noisy), dev(pre), dev(clean), flat)
    assert np.array_equal(host(g1), host(g2)) and np.array_equal(host(l1), host(l2))


def test_bf16_training_lowers_loss_and_is_faster():
    """Batch 64 of 64 x 64 crops, 40 steps from the same initial weights:
    the BF16 tensor-core steps lower the L1 loss as the FP32 steps do and take
    less time (CUDA events, after warm-up)."""
    import torch
    from paper_2403_03488_gb300 import api
    from paper_2403_03488_gb300.autograd import ResidualNet
    clean, noisy, pre = _case(6, 64, 64, 64)
    x, p, c = dev(noisy), dev(pre), dev(clean)
    res = {}
    for prec in (api.DN_FP32, api.DN_BF16):
        net = ResidualNet(10, 32, seed=6).cuda()
        losses = [net.train_step(x, p, c, precision=prec)]
        for _ in range(3):
            net.train_step(x, p, c, precision=prec, sync=False)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(36):
            net.train_step(x, p, c, precision=prec, sync=False)
        e1.record()
        e1.synchronize()
        losses.append(net.train_step(x, p, c, precision=prec))
        res[prec] = (losses, e0.elapsed_time(e1) / 36)
    print("training step, batch 64 x 64^2: FP32 %.2f ms, BF16 tensor cores %.2f ms; loss %.3f -> %.3f (FP32), "
          "%.3f -> %.3f (BF16)" % (res[api.DN_FP32][1], res[api.DN_BF16][1], res[api.DN_FP32][0][0],
                                  res[api.DN_FP32][0][-1], res[api.DN_BF16][0][0], res[api.DN_BF16][0][-1]))
    for prec in res:
        l0, l1 = res[prec][0][0], res[prec][0][-1]
        assert l1 < 0.9 * l0
    assert res[api.DN_BF16][0][-1] <= 1.05 * res[api.DN_FP32][0][-1]
    assert res[api.DN_BF16][1] < res[api.DN_FP32][1]
    assert api.device_error() == 0

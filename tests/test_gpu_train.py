"""The learned part (Sec. II, Eq. 2-3) on the library's kernels: the
autograd Function's gradients against finite differences and against the
FP64 oracle, one training step against the oracle's network gradients,
training lowering the L1 loss, and the trained network's gain over plain
BM3D on held-out scenes."""
import numpy as np
import pytest

from gpu_util import dev, host, need_gpu
from paper_2403_03488_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def test_conv3x3fn_gradients_finite_differences_and_oracle(oracle):
    import torch
    from paper_2403_03488_gb300.autograd import Conv3x3Fn
    rng = np.random.default_rng(0)
    x = torch.tensor(rng.normal(0, 1, (2, 3, 6, 7)), dtype=torch.float32, device="cuda", requires_grad=True)
    w = torch.tensor(rng.normal(0, 0.4, (4, 3, 3, 3)), dtype=torch.float32, device="cuda", requires_grad=True)
    b = torch.tensor(rng.normal(0, 0.1, 4), dtype=torch.float32, device="cuda", requires_grad=True)
    gy = torch.tensor(rng.normal(0, 1, (2, 4, 6, 7)), dtype=torch.float32, device="cuda")
    for relu in (False, True):
        for t in (x, w, b):
            t.grad = None
        y = Conv3x3Fn.apply(x, w, b, relu)
        (y * gy).sum().backward()
        # FP64 oracle of the same composition
        pre = oracle.conv3x3(host(x), host(w), host(b))
        g = host(gy) * (pre > 0) if relu else host(gy)
        dx, dw, db = oracle.conv3x3_bwd(host(x), g, host(w))
        np.testing.assert_allclose(host(x.grad), dx, atol=1e-4)
        np.testing.assert_allclose(host(w.grad), dw, atol=1e-3)
        np.testing.assert_allclose(host(b.grad), db, atol=1e-3)
        # central finite differences in FP32 on a few entries
        f = lambda: float((Conv3x3Fn.apply(x, w, b, relu) * gy).sum())
        eps = 1e-2
        with torch.no_grad():
            for t, idx in ((x, (1, 2, 3, 4)), (w, (2, 1, 0, 1)), (b, (3,))):
                old = float(t[idx])
                t[idx] = old + eps
                fp = f()
                t[idx] = old - eps
                fm = f()
                t[idx] = old
                num = (fp - fm) / (2 * eps)
                assert abs(num - float(t.grad[idx])) <= 2e-2 * max(1.0, abs(num))


def test_train_step_gradients_match_oracle(oracle):
    import torch
    from paper_2403_03488_gb300.autograd import ResidualNet
    rng = np.random.default_rng(1)
    clean = rng.uniform(0, 255, (3, 20, 24)).astype(np.float32)
    noisy = (clean + rng.normal(0, 25, clean.shape)).astype(np.float32)
    pre = (clean + rng.normal(0, 6, clean.shape)).astype(np.float32)
    net = ResidualNet(10, 32, seed=3).cuda()
    loss = net.train_step(dev(noisy), dev(pre), dev(clean))
    ref_loss, grads = oracle.cnn_backward(noisy, pre, clean, net.numpy_params_before_step())
    assert abs(loss - ref_loss) <= 1e-4 * max(1.0, ref_loss)
    for (gw, gb), (rw, rb) in zip(net.last_grads(), grads):
        gw, gb = host(gw), host(gb)
        assert np.abs(gw - rw).max() <= 1e-3 * max(1e-3, np.abs(rw).max())
        assert np.abs(gb - rb).max() <= 1e-3 * max(1e-3, np.abs(rb).max())


def test_training_lowers_the_l1_loss():
    from paper_2403_03488_gb300 import train
    net, hist = train.train(steps=300, batch=16, crop=48, n_images=8, log_every=100, log=lambda *_: None)
    assert hist[-1][1] < 0.9 * hist[0][1]


def test_trained_network_gains_over_bm3d():
    """Held-out scenes (seeds 5000+), never seen in training (seeds 10000+):
    the shipped trained weights add a clear PSNR gain to plain BM3D."""
    from paper_2403_03488_gb300 import serve, train
    w = serve.load_weights()
    res = train.evaluate(w, sigmas=(15.0, 25.0, 50.0), n_images=4, H=256, W=256)
    for s, r in res.items():
        assert r["gain_db"] > 0.3, (s, r)
        assert r["bm3d"] > r["noisy"] + 5.0

"""Pins of the oracle's NL-means and residual CNN.

NL-means: h -> inf gives the clipped search-window mean; h -> 0 keeps only the
candidates with d2 <= 2 sigma^2 (brute force with numpy's symmetric padding);
exact-duplicate scenes return their input.  CNN (Eq. 2-3): torch conv2d in
FP64 on the CPU, torch autograd, central finite differences, torch's Adam."""
import numpy as np
import pytest
import torch

from paper_2403_03488_gb300 import synth


def window_mean(y, search):
    H, W = y.shape
    hs = search // 2
    out = np.empty_like(y)
    for i in range(H):
        for j in range(W):
            out[i, j] = y[max(0, i - hs):i + hs + 1, max(0, j - hs):j + hs + 1].mean()
    return out


@pytest.mark.parametrize("H,W,search", [(13, 17, 21), (30, 25, 5), (6, 40, 21)])
def test_nlm_infinite_h_is_window_mean(oracle, H, W, search):
    y = np.random.default_rng(H).uniform(0, 255, (H, W))
    out = oracle.nlm(y, 25.0, patch=7, search=search, h=np.inf)
    np.testing.assert_allclose(out, window_mean(y, search), atol=1e-10)


def test_nlm_small_h_keeps_only_close_patches(oracle):
    """h -> 0: w = 1 where d2 <= 2 sigma^2, w = 0 otherwise (brute force with
    numpy's 'symmetric' padding, i.e. half-sample symmetric reflection)."""
    rng = np.random.default_rng(9)
    H, W, sigma = 14, 16, 20.0
    y = rng.uniform(0, 255, (H, W))
    y[:, 8:] = y[:, :8]  # exact repeats give close pairs
    y += rng.normal(0, 3, (H, W))
    yp = np.pad(y, 3, mode="symmetric")
    expect = np.empty_like(y)
    for i in range(H):
        for j in range(W):
            P = yp[i:i + 7, j:j + 7]
            acc = wsum = 0.0
            for qi in range(max(0, i - 10), min(H, i + 11)):
                for qj in range(max(0, j - 10), min(W, j + 11)):
                    d2 = ((P - yp[qi:qi + 7, qj:qj + 7]) ** 2).mean()
                    w = 1.0 if d2 <= 2 * sigma * sigma else 0.0
                    acc += w * y[qi, qj]
                    wsum += w
            expect[i, j] = acc / wsum
    out = oracle.nlm(y, sigma, h=1e-6)
    np.testing.assert_allclose(out, expect, atol=1e-9)


def test_nlm_brute_force_tiny(oracle):
    rng = np.random.default_rng(10)
    H, W, sigma = 11, 12, 15.0
    y = rng.uniform(0, 255, (H, W))
    h = 0.4 * sigma
    yp = np.pad(y, 3, mode="symmetric")
    expect = np.empty_like(y)
    for i in range(H):
        for j in range(W):
            P = yp[i:i + 7, j:j + 7]
            acc = wsum = 0.0
            for qi in range(max(0, i - 10), min(H, i + 11)):
                for qj in range(max(0, j - 10), min(W, j + 11)):
                    d2 = ((P - yp[qi:qi + 7, qj:qj + 7]) ** 2).mean()
                    w = np.exp(-max(d2 - 2 * sigma ** 2, 0.0) / h ** 2)
                    acc += w * y[qi, qj]
                    wsum += w
            expect[i, j] = acc / wsum
    np.testing.assert_allclose(oracle.nlm(y, sigma), expect, atol=1e-9)


def test_nlm_denoises(oracle):
    clean, noisy = synth.make_batch([1], 48, 48, 25.0)
    out = oracle.nlm(noisy[0, 0], 25.0)
    assert oracle.psnr(out, clean[0, 0]) > oracle.psnr(noisy[0, 0], clean[0, 0]) + 3.0


def _torch_conv(x, w, b):
    return torch.nn.functional.conv2d(torch.from_numpy(x), torch.from_numpy(w).permute(0, 3, 1, 2),
                                      None if b is None else torch.from_numpy(b), padding=1)


@pytest.mark.parametrize("N,Cin,Cout,H,W", [(2, 2, 32, 9, 11), (1, 32, 1, 7, 5), (3, 5, 4, 1, 6)])
def test_conv3x3_equals_torch_fp64(oracle, N, Cin, Cout, H, W):
    rng = np.random.default_rng(N + Cin)
    x = rng.normal(0, 1, (N, Cin, H, W))
    w = rng.normal(0, 0.3, (Cout, 3, 3, Cin))
    b = rng.normal(0, 0.1, Cout)
    np.testing.assert_allclose(oracle.conv3x3(x, w, b), _torch_conv(x, w, b).numpy(), atol=1e-12)


def test_conv3x3_bwd_equals_torch_autograd(oracle):
    rng = np.random.default_rng(3)
    x = rng.normal(0, 1, (2, 3, 6, 7))
    w = rng.normal(0, 0.3, (4, 3, 3, 3))
    b = rng.normal(0, 0.1, 4)
    dy = rng.normal(0, 1, (2, 4, 6, 7))
    xt = torch.from_numpy(x).requires_grad_()
    wt = torch.from_numpy(w).requires_grad_()
    bt = torch.from_numpy(b).requires_grad_()
    y = torch.nn.functional.conv2d(xt, wt.permute(0, 3, 1, 2), bt, padding=1)
    y.backward(torch.from_numpy(dy))
    dx, dw, db = oracle.conv3x3_bwd(x, dy, w)
    np.testing.assert_allclose(dx, xt.grad.numpy(), atol=1e-12)
    np.testing.assert_allclose(dw, wt.grad.numpy(), atol=1e-12)
    np.testing.assert_allclose(db, bt.grad.numpy(), atol=1e-12)


def test_conv3x3_bwd_finite_differences(oracle):
    rng = np.random.default_rng(4)
    x = rng.normal(0, 1, (1, 2, 5, 5))
    w = rng.normal(0, 0.3, (3, 3, 3, 2))
    dy = rng.normal(0, 1, (1, 3, 5, 5))
    dx, dw, _ = oracle.conv3x3_bwd(x, dy, w)
    f = lambda xx, ww: float((oracle.conv3x3(xx, ww) * dy).sum())
    eps = 1e-6
    for idx in [(0, 0, 0, 0), (0, 1, 2, 3), (0, 1, 4, 4)]:
        e = np.zeros_like(x)
        e[idx] = eps
        assert abs((f(x + e, w) - f(x - e, w)) / (2 * eps) - dx[idx]) < 1e-7
    for idx in [(0, 0, 0, 0), (2, 1, 2, 1), (1, 2, 0, 1)]:
        e = np.zeros_like(w)
        e[idx] = eps
        assert abs((f(x, w + e) - f(x, w - e)) / (2 * eps) - dw[idx]) < 1e-7


def test_cnn_backward_finite_differences(oracle):
    """Full residual network (2 layers, width 4) on a tiny crop: every gradient
    entry against central differences of the L1 loss of Eq. 2."""
    rng = np.random.default_rng(5)
    params = [(rng.normal(0, 0.5, (4, 3, 3, 2)), rng.normal(0, 0.1, 4)),
              (rng.normal(0, 0.5, (1, 3, 3, 4)), rng.normal(0, 0.1, 1))]
    clean = rng.uniform(0, 255, (2, 5, 6))
    noisy = clean + rng.normal(0, 25, clean.shape)
    pre = clean + rng.normal(0, 8, clean.shape)
    loss, grads = oracle.cnn_backward(noisy, pre, clean, params)
    eps = 1e-7
    for l, (w, b) in enumerate(params):
        for arr, g in ((w, grads[l][0]), (b, grads[l][1])):
            for i in range(arr.size):
                old = arr.flat[i]
                arr.flat[i] = old + eps
                lp = oracle.l1_loss(oracle.cnn_forward(noisy, pre, params), clean)
                arr.flat[i] = old - eps
                lm = oracle.l1_loss(oracle.cnn_forward(noisy, pre, params), clean)
                arr.flat[i] = old
                assert abs((lp - lm) / (2 * eps) - g.flat[i]) < 1e-6 * max(1.0, abs(g.flat[i]))


def test_cnn_forward_equals_torch_composition(oracle):
    rng = np.random.default_rng(6)
    params = synth.he_normal_weights(0, layers=3, width=8)
    noisy = rng.uniform(0, 255, (2, 9, 10))
    pre = rng.uniform(0, 255, (2, 9, 10))
    h = torch.from_numpy(np.stack([pre / 255.0, noisy / 255.0], axis=1))
    for l, (w, b) in enumerate(params):
        h = _torch_conv(h.numpy(), w.astype(np.float64), b.astype(np.float64))
        if l < 2:
            h = torch.relu(h)
    expect = pre + 255.0 * h[:, 0].numpy()
    np.testing.assert_allclose(oracle.cnn_forward(noisy, pre, params), expect, atol=1e-10)


def test_adam_equals_torch(oracle):
    rng = np.random.default_rng(7)
    p = rng.normal(0, 1, 10)
    pt = torch.tensor(p.copy(), requires_grad=True)
    opt = torch.optim.Adam([pt], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    for t in range(1, 4):
        g = rng.normal(0, 1, 10)
        opt.zero_grad()
        pt.grad = torch.tensor(g)
        opt.step()
        p, m, v = oracle.adam_step(p, g, m, v, t)
    np.testing.assert_allclose(p, pt.detach().numpy(), atol=1e-12)


def test_nlm_colour_weights_from_guide_channel(oracle):
    """Channels 1..C-1 are averaged with the weights of channel 0: a copy of the
    guide in channel 1 comes out equal to the guide's output, and a constant
    channel stays constant."""
    rng = np.random.default_rng(11)
    g = rng.uniform(0, 255, (12, 13))
    img = np.stack([g, g, np.full_like(g, 42.0)])
    out = oracle.nlm_channels(img, 20.0)
    np.testing.assert_allclose(out[1], out[0], atol=1e-12)
    np.testing.assert_allclose(out[2], 42.0, atol=1e-12)
    np.testing.assert_allclose(out[0], oracle.nlm(g, 20.0), atol=1e-12)


def test_cnn_forward_colour_native_block_diagonal_equals_grey_per_channel(oracle):
    """Eq. 3 on RGB: z = [pre R, G, B, noisy R, G, B] / 255.  A colour-native
    network whose weights never mix colour planes (layer 1 reads only planes
    c and 3 + c into hidden block c, hidden layers are block diagonal, the
    last layer writes block c to output c) must equal the grey network run on
    each plane -- an independent check of the channel order and of the
    per-plane residual."""
    rng = np.random.default_rng(4)
    grey = [(w * 0.7, rng.normal(0, 0.05, b.shape)) for w, b in synth.he_normal_weights(9, layers=4, width=4)]
    wd = 4
    colour = []
    for l, (w, b) in enumerate(grey):
        cout, _, _, cin = w.shape
        big_out = 3 if l == len(grey) - 1 else 3 * wd
        big_in = 6 if l == 0 else 3 * wd
        W = np.zeros((big_out, 3, 3, big_in))
        B = np.zeros(big_out)
        for c in range(3):
            oi = slice(c, c + 1) if l == len(grey) - 1 else slice(c * wd, (c + 1) * wd)
            if l == 0:
                W[oi, :, :, c] = w[:, :, :, 0]          # the pre plane of colour c
                W[oi, :, :, 3 + c] = w[:, :, :, 1]      # the noisy plane of colour c
            else:
                W[oi, :, :, c * wd:(c + 1) * wd] = w
            B[oi] = b
        colour.append((W, B))
    noisy = rng.uniform(0, 255, (2, 3, 11, 13))
    pre = noisy + rng.normal(0, 5, noisy.shape)
    out = oracle.cnn_forward(noisy, pre, colour)
    for c in range(3):
        ref = oracle.cnn_forward(noisy[:, c], pre[:, c], grey)
        np.testing.assert_allclose(out[:, c], ref, rtol=0, atol=1e-10)

"""Pins of the oracle of the flexible lightweight network (Sec. III): a
brute-force numpy definition of every layer and of the whole network (no
torch), finite differences of the gradients, the adjoint identity of the
transposed convolution, and the network's size against Table III."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402

WID = (2, 3, 2, 4, 3)


def shapes(c):
    out = []
    blocks = [(3, c[0]), (c[0], c[0])]
    for k in range(1, 5):
        blocks += [(c[k - 1], c[k]), (c[k], c[k])]
    spec = [("ds", a, b) for a, b in blocks]
    for k in range(4, 0, -1):
        spec += [("up", c[k], c[k - 1]), ("ds", c[k - 1], c[k - 1])]
    spec.append(("out", c[0], 1))
    for kind, a, b in spec:
        out += ([(a, 3, 3), (a,), (b, a), (b,)] if kind == "ds" else [(a, b, 2, 2), (b,)] if kind == "up"
                else [(1, a), (1,)])
    return out


def rand_params(c, seed):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal(s) * (0.5 if len(s) > 1 else 0.1) for s in shapes(c)]


def bf_dw(x, w, b, s):
    N, C, H, W = x.shape
    Ho, Wo = (H + s - 1) // s, (W + s - 1) // s
    xp = np.zeros((N, C, H + 2, W + 2))
    xp[:, :, 1:H + 1, 1:W + 1] = x
    y = np.zeros((N, C, Ho, Wo))
    for c in range(C):
        for yo in range(Ho):
            for xo in range(Wo):
                y[:, c, yo, xo] = b[c] + (w[c] * xp[:, c, s * yo:s * yo + 3, s * xo:s * xo + 3]).sum(axis=(1, 2))
    return y


def bf_pw(x, w, b):
    N, C, H, W = x.shape
    y = np.zeros((N, w.shape[0], H, W))
    for co in range(w.shape[0]):
        y[:, co] = b[co]
        for ci in range(C):
            y[:, co] += w[co, ci] * x[:, ci]
    return y


def bf_up(x, w, b):
    N, C, H, W = x.shape
    y = np.zeros((N, w.shape[1], 2 * H, 2 * W))
    for co in range(w.shape[1]):
        for i in range(H):
            for j in range(W):
                for a in range(2):
                    for d in range(2):
                        y[:, co, 2 * i + a, 2 * j + d] += (w[:, co, a, d] * x[:, :, i, j]).sum(axis=1)
        y[:, co] += b[co]
    return y


def bf_network(noisy, pre, sigma, params):
    N, H, W = noisy.shape
    h = np.stack([pre / 255.0, noisy / 255.0, np.broadcast_to(np.asarray(sigma)[:, None, None] / 255.0, (N, H, W))], 1)
    it = iter(params)

    def block(h, s):
        dw, db, pw, pb = next(it), next(it), next(it), next(it)
        return np.maximum(bf_pw(bf_dw(h, dw, db, s), pw, pb), 0.0)

    h = block(block(h, 1), 1)
    enc = [h]
    for _ in range(4):
        h = block(block(h, 2), 1)
        enc.append(h)
    for k in range(4, 0, -1):
        w, b = next(it), next(it)
        h = block(bf_up(h, w, b) + enc[k - 1], 1)
    w, b = next(it), next(it)
    return pre + 255.0 * bf_pw(h, w, b)[:, 0]


def test_oracle_network_equals_brute_force_definition():
    rng = np.random.default_rng(0)
    noisy = rng.uniform(0, 255, (2, 16, 32))
    pre = rng.uniform(0, 255, (2, 16, 32))
    prm = rand_params(WID, 1)
    out = oracle.fl_forward(noisy, pre, [25.0, 50.0], prm)
    ref = bf_network(noisy, pre, [25.0, 50.0], prm)
    np.testing.assert_allclose(out, ref, rtol=1e-11, atol=1e-9)


def test_oracle_network_gradients_by_finite_differences():
    rng = np.random.default_rng(2)
    noisy = rng.uniform(0, 255, (1, 16, 16))
    pre = noisy + rng.normal(0, 5, noisy.shape)
    clean = pre + rng.normal(0, 3, noisy.shape)
    prm = rand_params(WID, 3)
    loss, grads = oracle.fl_backward(noisy, pre, clean, [15.0], prm)
    h = 1e-6
    for t in range(14):
        li = int(rng.integers(0, len(prm)))
        idx = tuple(int(rng.integers(0, n)) for n in prm[li].shape)
        pp = [a.copy() for a in prm]
        pm = [a.copy() for a in prm]
        pp[li][idx] += h
        pm[li][idx] -= h
        lp = np.abs(oracle.fl_forward(noisy, pre, [15.0], pp) - clean).mean()
        lm = np.abs(oracle.fl_forward(noisy, pre, [15.0], pm) - clean).mean()
        fd = (lp - lm) / (2 * h)
        assert abs(fd - grads[li][idx]) <= 1e-5 * max(1.0, abs(fd)), (li, idx, fd, grads[li][idx])


def test_transposed_convolution_is_the_adjoint_of_the_strided_correlation():
    """<up(x), y> = <x, up^T(y)> with up^T(y)[ci][i][j] = sum_{co,a,c} w[ci][co][a][c] y[co][2i+a][2j+c]."""
    rng = np.random.default_rng(4)
    x = rng.standard_normal((1, 3, 5, 4))
    w = rng.standard_normal((3, 2, 2, 2))
    y = rng.standard_normal((1, 2, 10, 8))
    up = bf_up(x, w, np.zeros(2))
    adj = np.zeros_like(x)
    for a in range(2):
        for c in range(2):
            adj += np.einsum("iocd,nohw->nihw", w[:, :, a:a + 1, c:c + 1], y[:, :, a::2, c::2])
    assert abs((up * y).sum() - (x * adj).sum()) < 1e-10 * abs((up * y).sum()) + 1e-12
    # and the oracle's transposed convolution is the same operator
    torch_, F = oracle._fl_torch()
    t = F.conv_transpose2d(torch.as_tensor(x), torch.as_tensor(w), stride=2).numpy()
    np.testing.assert_allclose(t, up, rtol=1e-12, atol=1e-12)


def test_network_size_matches_table_III():
    """The widths chosen for the unpublished block details give the paper's
    compute: 4.52 GMAC per 512 x 512 image (Table III)."""
    from paper_2403_03488_gb300 import flnet
    g = flnet.macs_per_pixel() * 512 * 512 / 1e9
    assert abs(g - 4.52) / 4.52 < 0.01, g
    # the closed form agrees with a layer-by-layer count of the spec
    c = flnet.WIDTHS
    n = 0.0
    res = 1.0
    for kind, cin, cout, s in flnet.layer_specs():
        if kind == "ds":
            res = res / 4 if s == 2 else res
            n += res * (9 * cin + cin * cout)
        elif kind == "up":
            res *= 4
            n += res * cin * cout
        else:
            n += cin
    assert abs(n - flnet.macs_per_pixel()) < 1e-6
    assert len(flnet.param_shapes()) == len(shapes(c))
    assert all(tuple(a) == tuple(b) for a, b in zip(flnet.param_shapes(), shapes(c)))


def test_work_per_pixel_splits_the_network_count():
    """The per-kind counts the roofline uses add up to the whole network's
    multiply-adds, and the depthwise bytes match a count on explicit plane sizes
    (a 1024 x 1024 image, planes read once and written once)."""
    from paper_2403_03488_gb300 import flnet
    w = flnet.work_per_pixel()
    assert abs(w["dw_macs"] + w["pw_macs"] + w["up_macs"] - flnet.macs_per_pixel()) < 1e-9
    side, b = 1024, 0
    for kind, cin, cout, s in flnet.layer_specs():
        if kind == "ds":
            out = side // s
            b += 4 * cin * (side * side + out * out)
            side = out
        elif kind == "up":
            side *= 2
    assert abs(b / 1024 ** 2 - w["dw_bytes"]) < 1e-9

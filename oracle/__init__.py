"""FP64 oracle of the nonlocal + neural denoiser -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg (and its
reference arm) may import this package.  The product path (the CUDA library
and its binding) never imports it, and it imports nothing from the product.

Layout: the slow C restatement in oracle.c (built into _oracle.so by
build()), wrapped here with numpy; the colour transform, the network
composition of Eq. 2-3, the L1 loss, Adam and PSNR are plain numpy.

Pins: every function here is checked by tests/test_oracle_*.py against
library routines (scipy DCT, scipy Hadamard, numpy Kaiser, torch conv2d in
FP64), closed forms (lambda3D = 0 identity, constant-image fixed point,
NLM with h -> inf equals the window mean, repeated-tile matches), brute force
on tiny images and finite differences.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (OpenMP, no FP contraction)."""
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        cmd = ["gcc", "-O2", "-std=gnu99", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-o", _SO + ".tmp", src, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_SO + ".tmp", _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        up = ctypes.POINTER(ctypes.c_ubyte)
        i, d = ctypes.c_int, ctypes.c_double
        L.or_dct8.argtypes = [dp]
        L.or_dct.argtypes = [i, dp]
        L.or_dct2d_matrix.argtypes = [dp]
        L.or_dct2d_matrix_k.argtypes = [i, dp]
        L.or_hadamard.argtypes = [i, dp]
        L.or_kaiser.argtypes = [i, d, dp]
        L.or_t3d.argtypes = [dp, i, i, dp]
        L.or_t3d_k.argtypes = [dp, i, i, i, dp]
        L.or_grid.argtypes = [i, i, i, ip]
        L.or_match.argtypes = [dp, i, i, i, i, i, i, d, ip, dp, ip, ip, up]
        L.or_match_pre.argtypes = [dp, i, i, i, i, i, i, d, d, d, d, d, ip, dp, ip, ip, up]
        L.or_bm3d_pass1.argtypes = [dp, i, i, i, dp, i, i, i, i, d, d, d, d, d, d, dp, up, up]
        L.or_bm3d_pass2.argtypes = [dp, dp, i, i, i, dp, i, i, i, i, d, d, dp, up, up]
        L.or_nlm.argtypes = [dp, i, i, i, d, i, i, d, dp]
        L.or_conv3x3.argtypes = [dp, i, i, i, i, dp, dp, i, dp]
        L.or_conv3x3_bwd.argtypes = [dp, dp, i, i, i, i, dp, i, dp, dp, dp]
        L.or_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _dp(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _up(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return lib().or_num_threads()


# --------------------------------------------------------------------------
# Transforms and windows (exported for the pins)
# --------------------------------------------------------------------------

def dct8() -> np.ndarray:
    C = np.empty((8, 8))
    lib().or_dct8(_dp(C))
    return C


def dct(k: int) -> np.ndarray:
    """Orthonormal DCT-II matrix of size k (rows = frequencies)."""
    C = np.empty((k, k))
    lib().or_dct(k, _dp(C))
    return C


def dct2d_matrix(k: int = 8) -> np.ndarray:
    """The 2D DCT of a k x k patch as a k^2 x k^2 matrix on the row-major patch."""
    T = np.empty((k * k, k * k))
    if k == 8:
        lib().or_dct2d_matrix(_dp(T))
    else:
        lib().or_dct2d_matrix_k(k, _dp(T))
    return T


def hadamard(n: int) -> np.ndarray:
    Hm = np.empty((n, n))
    if lib().or_hadamard(n, _dp(Hm)):
        raise ValueError("n must be a power of two <= 64")
    return Hm


def kaiser(M: int, beta: float) -> np.ndarray:
    w = np.empty(M)
    lib().or_kaiser(M, beta, _dp(w))
    return w


def t3d(G: np.ndarray, inverse: bool = False) -> np.ndarray:
    """3D transform of a group G [n, k*k] (2D DCT per k x k patch, Hadamard
    along n); k = 8 for 64 columns."""
    G = _f64(G)
    Z = np.empty_like(G)
    k = int(round(np.sqrt(G.shape[1])))
    if k * k != G.shape[1]:
        raise ValueError("patches must be square")
    rc = (lib().or_t3d(_dp(G), G.shape[0], int(inverse), _dp(Z)) if k == 8
          else lib().or_t3d_k(_dp(G), G.shape[0], k, int(inverse), _dp(Z)))
    if rc:
        raise ValueError("bad group or patch size")
    return Z


def grid(L: int, k: int = 8, step: int = 3) -> np.ndarray:
    n = lib().or_grid(L, k, step, None)
    pos = np.zeros(max(n, 1), np.int32)
    lib().or_grid(L, k, step, _ip(pos))
    return pos[:n]


# --------------------------------------------------------------------------
# BM3D
# --------------------------------------------------------------------------

FLAG_TAU, FLAG_TIE, FLAG_THR, FLAG_PRE = 1, 2, 4, 8
LAMBDA2D_HIGH = 2.0  # 2D prethreshold of the first-pass distance above sigma 40 (regime 0)
PRE_BAND = 0.005     # hazard band of the prethreshold decision (absolute, 0..255 scale)


@dataclass
class Pass:
    """Parameters of one BM3D pass (standard BM3D notation)."""
    patch: int = 8
    step: int = 3
    search: int = 39
    n2: int = 16
    tau: float = 2500.0
    lambda3d: float = 2.7
    beta: float = 2.0
    lambda2d: float = 0.0  # > 0: first-pass distances on 2D-prethresholded patches (threshold lambda2d * sigma)


def default_passes(sigma: float, regime: int = 0):
    """(hard, wiener) parameters.  regime 0: tau1 = 2500, tau2 = 400 for
    sigma <= 40; above, tau1 = 5000, tau2 = 3500 and the first pass matches on
    2D-prethresholded patches (lambda2d = 2); regime 1: 2500 / 400 and raw
    patches always."""
    hi = regime == 0 and sigma > 40.0
    return (Pass(n2=16, tau=5000.0 if hi else 2500.0, lambda2d=LAMBDA2D_HIGH if hi else 0.0),
            Pass(n2=32, tau=3500.0 if hi else 400.0))


def match(guide: np.ndarray, p: Pass):
    """Exhaustive block matching on one [H, W] guide.

    Returns dict(idx [Ry, Rx, n2] int32, dist [Ry, Rx, n2+1], nkept, n, flag)."""
    g = _f64(guide)
    H, W = g.shape
    Ry, Rx = len(grid(H, p.patch, p.step)), len(grid(W, p.patch, p.step))
    R = Ry * Rx
    idx = np.empty((R, p.n2), np.int32)
    dist = np.empty((R, p.n2 + 1))
    nk = np.empty(R, np.int32)
    ng = np.empty(R, np.int32)
    fl = np.empty(R, np.uint8)
    rc = lib().or_match(_dp(g), H, W, p.patch, p.step, p.search, p.n2, p.tau,
                        _ip(idx), _dp(dist), _ip(nk), _ip(ng), _up(fl))
    if rc:
        raise ValueError("or_match: bad arguments")
    return dict(idx=idx.reshape(Ry, Rx, p.n2), dist=dist.reshape(Ry, Rx, p.n2 + 1),
                nkept=nk.reshape(Ry, Rx), n=ng.reshape(Ry, Rx), flag=fl.reshape(Ry, Rx))


def match_pre(guide: np.ndarray, p: Pass, thr: float, band: float = PRE_BAND, rtie: float = 1e-5,
              atie: float = 1e-3):
    """Block matching on 2D-prethresholded patches (threshold thr) of one
    [H, W] guide; same outputs as `match`, flags including FLAG_PRE.  Ties:
    |a - b| <= rtie max(a, b) + atie (sqrt(a) + sqrt(b)) (atie = 1e-3 covers
    coefficient differences off by up to 5e-4, the FP32 transforms' error)."""
    g = _f64(guide)
    H, W = g.shape
    Ry, Rx = len(grid(H, p.patch, p.step)), len(grid(W, p.patch, p.step))
    R = Ry * Rx
    idx = np.empty((R, p.n2), np.int32)
    dist = np.empty((R, p.n2 + 1))
    nk = np.empty(R, np.int32)
    ng = np.empty(R, np.int32)
    fl = np.empty(R, np.uint8)
    rc = lib().or_match_pre(_dp(g), H, W, p.patch, p.step, p.search, p.n2, p.tau, float(thr), float(band),
                            float(rtie), float(atie), _ip(idx), _dp(dist), _ip(nk), _ip(ng), _up(fl))
    if rc:
        raise ValueError("or_match_pre: bad arguments (%d)" % rc)
    return dict(idx=idx.reshape(Ry, Rx, p.n2), dist=dist.reshape(Ry, Rx, p.n2 + 1),
                nkept=nk.reshape(Ry, Rx), n=ng.reshape(Ry, Rx), flag=fl.reshape(Ry, Rx))


def pass1_matches(guide: np.ndarray, p: Pass, sig_guide: float):
    """The match lists `bm3d_pass1` groups with: on 2D-prethresholded patches
    (threshold p.lambda2d * sig_guide) when p.lambda2d > 0, on pixels otherwise."""
    if p.lambda2d > 0.0:
        return match_pre(guide, p, p.lambda2d * float(sig_guide))
    return match(guide, p)


def bm3d_pass1(img: np.ndarray, sig, p: Pass, band: float = 0.0):
    """First pass on [C, H, W] (channel 0 guides matching).  Returns
    (basic [C, H, W], pixel flags [H, W], group flags [Ry, Rx])."""
    x = _f64(img)
    C, H, W = x.shape
    s = _f64(np.broadcast_to(np.asarray(sig, np.float64), (C,)))
    out = np.empty_like(x)
    pf = np.empty((H, W), np.uint8)
    Ry, Rx = len(grid(H, p.patch, p.step)), len(grid(W, p.patch, p.step))
    gf = np.empty((Ry, Rx), np.uint8)
    rc = lib().or_bm3d_pass1(_dp(x), C, H, W, _dp(s), p.patch, p.step, p.search, p.n2, p.tau,
                             p.lambda3d, p.beta, band, p.lambda2d * float(s[0]), PRE_BAND, _dp(out), _up(pf),
                             _up(gf))
    if rc:
        raise ValueError("or_bm3d_pass1 failed (%d)" % rc)
    return out, pf, gf


def bm3d_pass2(noisy: np.ndarray, basic: np.ndarray, sig, p: Pass):
    """Second pass on [C, H, W] given the basic estimate.  Returns
    (final [C, H, W], pixel flags [H, W], group flags [Ry, Rx])."""
    y = _f64(noisy)
    b = _f64(basic)
    C, H, W = y.shape
    s = _f64(np.broadcast_to(np.asarray(sig, np.float64), (C,)))
    out = np.empty_like(y)
    pf = np.empty((H, W), np.uint8)
    Ry, Rx = len(grid(H, p.patch, p.step)), len(grid(W, p.patch, p.step))
    gf = np.empty((Ry, Rx), np.uint8)
    rc = lib().or_bm3d_pass2(_dp(y), _dp(b), C, H, W, _dp(s), p.patch, p.step, p.search, p.n2,
                             p.tau, p.beta, _dp(out), _up(pf), _up(gf))
    if rc:
        raise ValueError("or_bm3d_pass2 failed (%d)" % rc)
    return out, pf, gf


# Full-range BT.601 RGB -> YCbCr rows (offsets drop out of the filter).
YCC = np.array([[0.299, 0.587, 0.114],
                [-0.168736, -0.331264, 0.5],
                [0.5, -0.418688, -0.081312]])


def rgb_to_ycc(x: np.ndarray) -> np.ndarray:
    return np.einsum("ij,jhw->ihw", YCC, _f64(x))


def ycc_to_rgb(x: np.ndarray) -> np.ndarray:
    return np.einsum("ij,jhw->ihw", np.linalg.inv(YCC), _f64(x))


def channel_sigmas(sigma: float, C: int) -> np.ndarray:
    """Per-channel noise std after the colour transform: sigma * ||row||_2."""
    if C == 1:
        return np.array([float(sigma)])
    return float(sigma) * np.sqrt((YCC ** 2).sum(axis=1))


def bm3d(noisy: np.ndarray, sigma: float, regime: int = 0, hard: Pass = None, wiener: Pass = None):
    """Both BM3D passes on one [C, H, W] image (C in {1, 3}); colour images are
    matched on Y and filtered per YCbCr channel.  Returns (basic, final) in
    the input colour space."""
    C = noisy.shape[0]
    dh, dw = default_passes(sigma, regime)
    hard = hard or dh
    wiener = wiener or dw
    x = rgb_to_ycc(noisy) if C == 3 else _f64(noisy)
    s = channel_sigmas(sigma, C)
    basic, _, _ = bm3d_pass1(x, s, hard)
    final, _, _ = bm3d_pass2(x, basic, s, wiener)
    if C == 3:
        return ycc_to_rgb(basic), ycc_to_rgb(final)
    return basic, final


# --------------------------------------------------------------------------
# NL-means
# --------------------------------------------------------------------------

def nlm_channels(img: np.ndarray, sigma: float, patch: int = 7, search: int = 21, h: float = None,
                 h_over_sigma: float = 0.4) -> np.ndarray:
    """NL-means of [C, H, W] with weights from channel 0 (the guide), applied to
    every channel; h defaults to h_over_sigma * sigma (sigma of the guide)."""
    y = _f64(img)
    C, H, W = y.shape
    out = np.empty_like(y)
    hh = float(h_over_sigma * sigma) if h is None else float(h)
    if lib().or_nlm(_dp(y), C, H, W, float(sigma), patch, search, hh, _dp(out)):
        raise ValueError("or_nlm: bad arguments")
    return out


def nlm(noisy: np.ndarray, sigma: float, patch: int = 7, search: int = 21, h_over_sigma: float = 0.4,
        h: float = None) -> np.ndarray:
    """Pixel-wise NL-means of one [H, W] image."""
    return nlm_channels(_f64(noisy)[None], sigma, patch, search, h, h_over_sigma)[0]


def nlm_image(noisy: np.ndarray, sigma: float, patch: int = 7, search: int = 21,
              h_over_sigma: float = 0.4) -> np.ndarray:
    """NL-means of one [C, H, W] image (C in {1, 3}).  Colour images are
    filtered in YCbCr with weights from Y (noise std sigma_Y) and converted back."""
    C = noisy.shape[0]
    if C == 1:
        return nlm_channels(noisy, sigma, patch, search, h_over_sigma=h_over_sigma)
    s = channel_sigmas(sigma, 3)[0]
    return ycc_to_rgb(nlm_channels(rgb_to_ycc(noisy), s, patch, search, h_over_sigma=h_over_sigma))


# --------------------------------------------------------------------------
# Residual CNN (Eq. 2-3)
# --------------------------------------------------------------------------

def conv3x3(x: np.ndarray, w: np.ndarray, b: np.ndarray = None) -> np.ndarray:
    """x [N, Cin, H, W], w [Cout, 3, 3, Cin], b [Cout] -> [N, Cout, H, W]."""
    x = _f64(x)
    w = _f64(w)
    N, Cin, H, W = x.shape
    Cout = w.shape[0]
    y = np.empty((N, Cout, H, W))
    lib().or_conv3x3(_dp(x), N, Cin, H, W, _dp(w), _dp(None if b is None else _f64(b)), Cout, _dp(y))
    return y


def conv3x3_bwd(x: np.ndarray, dy: np.ndarray, w: np.ndarray):
    """(dx, dw, db) of conv3x3 given dy."""
    x = _f64(x)
    dy = _f64(dy)
    w = _f64(w)
    N, Cin, H, W = x.shape
    Cout = w.shape[0]
    dx = np.empty_like(x)
    dw = np.empty_like(w)
    db = np.empty(Cout)
    lib().or_conv3x3_bwd(_dp(x), _dp(dy), N, Cin, H, W, _dp(w), Cout, _dp(dx), _dp(dw), _dp(db))
    return dx, dw, db


def cnn_forward(noisy: np.ndarray, pre: np.ndarray, params, keep: bool = False):
    """Residual CNN (Eq. 2-3).

    noisy, pre: [N, H, W] single-channel planes, or [N, cc, H, W] for a
    colour-native network (pre = BM3D or NLM output), 0..255 scale.
    z = [pre / 255, noisy / 255] (all pre planes, then all noisy planes);
    K-1 conv+bias+ReLU layers and a final conv+bias with cc outputs;
    output = pre + 255 * r.  params: list of (W [Cout,3,3,Cin], b).
    With keep=True also returns the layer inputs and pre-activations."""
    colour = np.ndim(noisy) == 4
    p4 = _f64(pre) if colour else _f64(pre)[:, None]
    n4 = _f64(noisy) if colour else _f64(noisy)[:, None]
    z = np.concatenate([p4 / 255.0, n4 / 255.0], axis=1)
    acts, pres = [z], []
    h = z
    for l, (w, b) in enumerate(params):
        a = conv3x3(h, w, b)
        pres.append(a)
        h = np.maximum(a, 0.0) if l < len(params) - 1 else a
        acts.append(h)
    out = p4 + 255.0 * h
    out = out if colour else out[:, 0]
    if keep:
        return out, acts, pres
    return out


def l1_loss(out: np.ndarray, clean: np.ndarray) -> float:
    """L = 1/N sum |x - (F(z) + BM3D(y))| (Eq. 2), N = number of pixels."""
    return float(np.mean(np.abs(_f64(clean) - _f64(out))))


def cnn_backward(noisy, pre, clean, params):
    """Gradients of l1_loss(cnn_forward(...)) w.r.t. every (W, b).

    dL/dout = sign(out - x) / N (0 where equal); dL/dr = 255 dL/dout."""
    out, acts, pres = cnn_forward(noisy, pre, params, keep=True)
    N = out.size
    g_out = np.sign(out - _f64(clean)) / N
    g = (255.0 * g_out)[:, None]
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        if l < len(params) - 1:
            g = g * (pres[l] > 0)
        dx, dw, db = conv3x3_bwd(acts[l], g, params[l][0])
        grads[l] = (dw, db)
        g = dx
    return l1_loss(out, clean), grads


def adam_step(param, grad, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba), bias-corrected; returns (param, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return param - lr * mh / (np.sqrt(vh) + eps), m, v


# --------------------------------------------------------------------------
# Flexible lightweight network (Sec. III, "Ours-FL")
# --------------------------------------------------------------------------
#
# Read from Sec. III: a U-Net of 4 encoder and 4 decoder levels built from 3x3
# depthwise-separable convolutions (depthwise 3x3 with bias, pointwise with
# bias, ReLU), a stride-2 block for every downsampling, a 2x2 stride-2
# transposed convolution plus the encoder output of the same level for every
# upsampling, a noise-level plane in the input (FFDNet style) and the
# residual output of Eq. 2.  Parameter order (the interface shared with the
# GPU network): per block dw_w [cin,3,3], dw_b, pw_w [cout,cin], pw_b; per
# upsampling w [cin,cout,2,2], b; then the output pw w [1,c0], b [1].  Plain
# PyTorch CPU ops in FP64 (grouped conv2d, conv_transpose2d, autograd), pinned
# in tests/test_oracle_flnet.py by brute-force numpy definitions, the adjoint
# identity of the transposed convolution and finite differences.

def _fl_torch():
    import torch
    import torch.nn.functional as F
    return torch, F


def fl_residual_t(noisy, pre, sigma, params):
    """The network's residual r [N, H, W] as a float64 torch tensor (params:
    float64 torch tensors, may require grad)."""
    torch, F = _fl_torch()
    nz = torch.as_tensor(_f64(noisy))
    pr = torch.as_tensor(_f64(pre))
    N, H, W = nz.shape
    sig = torch.as_tensor(np.asarray(sigma, np.float64).reshape(N, 1, 1) / 255.0).expand(N, H, W)
    h = torch.stack([pr / 255.0, nz / 255.0, sig], dim=1)
    it = iter(params)

    def block(h, stride):
        dw_w, dw_b, pw_w, pw_b = next(it), next(it), next(it), next(it)
        C = h.shape[1]
        h = F.conv2d(h, dw_w.reshape(C, 1, 3, 3), dw_b, stride=stride, padding=1, groups=C)
        h = F.conv2d(h, pw_w.reshape(pw_w.shape[0], C, 1, 1), pw_b)
        return torch.relu(h)

    h = block(block(h, 1), 1)
    enc = [h]
    for _ in range(4):
        h = block(block(h, 2), 1)
        enc.append(h)
    for k in range(4, 0, -1):
        w, b = next(it), next(it)
        h = F.conv_transpose2d(h, w, b, stride=2) + enc[k - 1]
        h = block(h, 1)
    w, b = next(it), next(it)
    r = F.conv2d(h, w.reshape(1, -1, 1, 1), b)
    return r[:, 0]


def fl_forward(noisy, pre, sigma, params):
    """out = pre + 255 r (numpy float64)."""
    torch, _ = _fl_torch()
    p = [torch.as_tensor(_f64(a)) for a in params]
    r = fl_residual_t(noisy, pre, sigma, p)
    return _f64(pre) + 255.0 * r.numpy()


def fl_backward(noisy, pre, clean, sigma, params):
    """(L1 loss of Eq. 2, gradients of every parameter) in float64."""
    torch, _ = _fl_torch()
    p = [torch.as_tensor(_f64(a)).requires_grad_(True) for a in params]
    r = fl_residual_t(noisy, pre, sigma, p)
    out = torch.as_tensor(_f64(pre)) + 255.0 * r
    loss = (out - torch.as_tensor(_f64(clean))).abs().mean()
    loss.backward()
    return float(loss.detach()), [q.grad.numpy() for q in p]


# --------------------------------------------------------------------------
# Error metrics
# --------------------------------------------------------------------------

def psnr(out: np.ndarray, clean: np.ndarray, peak: float = 255.0) -> float:
    """(C)PSNR of the output clipped to [0, peak]: MSE over every pixel and channel."""
    e = np.clip(_f64(out), 0.0, peak) - _f64(clean)
    mse = float(np.mean(e * e))
    return float("inf") if mse == 0 else 10.0 * np.log10(peak * peak / mse)

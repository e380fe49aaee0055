"""Torch-facing binding of the C ABI: same names as include/denoise.h.

Each function validates tensor placement, dtype and layout, allocates the
outputs and the workspace with PyTorch (device memory only), and calls the
library on the current CUDA stream.  Nothing here computes.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import torch

from . import _lib as L
from ._lib import (BM3DParams, BM3DPass, CNN, DN_BF16, DN_BF16_MATCH, DN_FP32, DN_PREFILTER_BM3D,
                   DN_PREFILTER_NLM, NLMParams, check, default_bm3d_params, default_nlm_params, farr)

__all__ = ["denoise_bm3d", "denoise_nlm", "denoise_hybrid", "bm3d_match", "bm3d_filter_hard", "bm3d_filter_wiener",
           "rgb_to_ycc", "ycc_to_rgb", "error_reduce", "conv3x3_fwd", "conv3x3_bwd_data", "conv3x3_bwd_weight",
           "cnn_forward", "l1_residual_grad", "adam_step", "grid", "default_bm3d_params", "default_nlm_params",
           "cnn_param_count", "profile", "bm3d_halo", "denoise_bm3d_tiled", "cnn_grad", "DN_FP32", "DN_BF16", "DN_BF16_MATCH",
           "DN_PREFILTER_BM3D", "DN_PREFILTER_NLM"]


def _vp(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _need(t: torch.Tensor, name: str, dtype=torch.float32, dim=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise ValueError("%s must be %s" % (name, dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if dim is not None and t.dim() != dim:
        raise ValueError("%s must have %d dimensions" % (name, dim))


def _ws(nbytes: int, device, workspace: Optional[torch.Tensor]):
    if nbytes == 0:
        return None, 0
    if workspace is not None:
        _need(workspace, "workspace", torch.uint8)
        if workspace.numel() < nbytes:
            raise ValueError("workspace too small: %d < %d bytes" % (workspace.numel(), nbytes))
        return workspace, workspace.numel()
    return torch.empty(nbytes, dtype=torch.uint8, device=device), nbytes


def _sigmas(sigma, B):
    s = [float(sigma)] * B if isinstance(sigma, (int, float)) else [float(v) for v in sigma]
    if len(s) != B:
        raise ValueError("need one sigma per image")
    return farr(s)


def grid(L_: int, patch: int = 8, step: int = 3):
    n = L.lib().dn_bm3d_grid(L_, patch, step, None)
    pos = (ctypes.c_int * max(n, 1))()
    L.lib().dn_bm3d_grid(L_, patch, step, pos)
    return list(pos)[:n]


def cnn_param_count(layers: int = 10, width: int = 32, channels: int = 1) -> int:
    """Floats in a weight buffer; channels = 3 for a colour-native network."""
    return int(L.lib().dn_cnn_param_count_c(layers, width, channels))


def bm3d_workspace_bytes(B, C, H, W, params: BM3DParams) -> int:
    return int(L.lib().dn_bm3d_workspace_bytes(B, C, H, W, ctypes.byref(params)))


def denoise_bm3d(noisy: torch.Tensor, sigma, params: Optional[BM3DParams] = None, out=None, workspace=None,
                 stream=None) -> torch.Tensor:
    """Both BM3D passes on [B, C, H, W] float32 (0..255); sigma per image."""
    _need(noisy, "noisy", dim=4)
    B, C, H, W = noisy.shape
    p = params or default_bm3d_params()
    out = torch.empty_like(noisy) if out is None else out
    _need(out, "out", dim=4)
    ws, nb = _ws(bm3d_workspace_bytes(B, C, H, W, p), noisy.device, workspace)
    check(L.lib().denoise_bm3d(_vp(noisy), _vp(out), B, C, H, W, _sigmas(sigma, B), ctypes.byref(p), _vp(ws), nb,
                               _stream(stream)), "denoise_bm3d")
    return out




def noalloc_scratch_bytes() -> int:
    """Size of the fixed device array behind denoise_bm3d_noalloc, as built."""
    return int(L.lib().dn_noalloc_scratch_bytes())


def denoise_bm3d_noalloc(noisy: torch.Tensor, sigma, params: Optional[BM3DParams] = None, out=None,
                         stream=None) -> torch.Tensor:
    """denoise_bm3d whose workspace is the library's own fixed device array
    (noalloc_scratch_bytes() bytes), for callers that may not allocate device
    memory.  Calls on one device share that array: do not let them overlap.
    (This wrapper still allocates `out` with torch when it is not given.)"""
    _need(noisy, "noisy", dim=4)
    B, C, H, W = noisy.shape
    p = params or default_bm3d_params()
    out = torch.empty_like(noisy) if out is None else out
    _need(out, "out", dim=4)
    check(L.lib().denoise_bm3d_noalloc(_vp(noisy), _vp(out), B, C, H, W, _sigmas(sigma, B), ctypes.byref(p),
                                       _stream(stream)), "denoise_bm3d_noalloc")
    return out


def bm3d_halo(params: Optional[BM3DParams] = None) -> int:
    """Pixels (per axis) an output pixel of BM3D depends on: the halo of a tile."""
    return int(L.lib().dn_bm3d_halo(ctypes.byref(params or default_bm3d_params())))


def denoise_bm3d_tiled(noisy: torch.Tensor, sigma: float, params: Optional[BM3DParams] = None, tile: int = 512,
                       max_batch: int = 4, out=None, workspace=None, stream=None) -> torch.Tensor:
    """BM3D of one [C, H, W] image in tiles of tile x tile pixels plus the halo
    (bit-identical to denoise_bm3d on the whole image)."""
    _need(noisy, "noisy", dim=3)
    C, H, W = noisy.shape
    p = params or default_bm3d_params()
    out = torch.empty_like(noisy) if out is None else out
    _need(out, "out", dim=3)
    nbytes = int(L.lib().dn_bm3d_tiled_workspace_bytes(C, H, W, ctypes.byref(p), tile, max_batch))
    ws, nb = _ws(nbytes, noisy.device, workspace)
    check(L.lib().denoise_bm3d_tiled(_vp(noisy), _vp(out), C, H, W, float(sigma), ctypes.byref(p), tile, max_batch,
                                     _vp(ws), nb, _stream(stream)), "denoise_bm3d_tiled")
    return out


def denoise_nlm(noisy: torch.Tensor, sigma, params: Optional[NLMParams] = None, out=None, workspace=None,
                stream=None) -> torch.Tensor:
    _need(noisy, "noisy", dim=4)
    B, C, H, W = noisy.shape
    p = params or default_nlm_params()
    out = torch.empty_like(noisy) if out is None else out
    _need(out, "out", dim=4)
    ws, nb = _ws(int(L.lib().dn_nlm_workspace_bytes(B, C, H, W, ctypes.byref(p))), noisy.device, workspace)
    check(L.lib().denoise_nlm(_vp(noisy), _vp(out), B, C, H, W, _sigmas(sigma, B), ctypes.byref(p), _vp(ws), nb,
                              _stream(stream)), "denoise_nlm")
    return out


def make_cnn(weights: torch.Tensor, layers: int = 10, width: int = 32, precision: int = DN_FP32,
             channels: int = 1) -> CNN:
    _need(weights, "weights", dim=1)
    if weights.numel() != cnn_param_count(layers, width, channels):
        raise ValueError("weights must hold %d floats" % cnn_param_count(layers, width, channels))
    return CNN(layers, width, ctypes.c_void_p(weights.data_ptr()), precision, channels)


def hybrid_workspace_bytes(B, C, H, W, prefilter, pparams, cnn: CNN) -> int:
    return int(L.lib().dn_hybrid_workspace_bytes(B, C, H, W, prefilter, ctypes.cast(ctypes.byref(pparams), ctypes.c_void_p),
                                                 ctypes.byref(cnn)))


def denoise_hybrid(noisy: torch.Tensor, sigma, weights: torch.Tensor, layers: int = 10, width: int = 32,
                   prefilter: int = DN_PREFILTER_BM3D, prefilter_params=None, cnn_precision: int = DN_FP32,
                   out=None, workspace=None, stream=None, cnn_channels: int = 1) -> torch.Tensor:
    """Nonlocal prefilter then the residual CNN (Eq. 2-3); cnn_channels = 3
    selects a colour-native network for RGB input."""
    _need(noisy, "noisy", dim=4)
    B, C, H, W = noisy.shape
    if prefilter_params is None:
        prefilter_params = default_bm3d_params() if prefilter == DN_PREFILTER_BM3D else default_nlm_params()
    cnn = make_cnn(weights, layers, width, cnn_precision, cnn_channels)
    out = torch.empty_like(noisy) if out is None else out
    _need(out, "out", dim=4)
    ws, nb = _ws(hybrid_workspace_bytes(B, C, H, W, prefilter, prefilter_params, cnn), noisy.device, workspace)
    check(L.lib().denoise_hybrid(_vp(noisy), _vp(out), B, C, H, W, _sigmas(sigma, B), prefilter,
                                 ctypes.cast(ctypes.byref(prefilter_params), ctypes.c_void_p), ctypes.byref(cnn),
                                 _vp(ws), nb, _stream(stream)), "denoise_hybrid")
    return out


def bm3d_match(guide: torch.Tensor, tau, p: BM3DPass, precision: int = DN_FP32, stream=None):
    """guide [B, H, W] (or a [B, C, H, W] image, matched on channel 0).
    Returns (idx int32 [B, Ry, Rx, n2], n int32 [B, Ry, Rx])."""
    if guide.dim() == 4:
        B, C, H, W = guide.shape
        plane = C * H * W
    else:
        B, H, W = guide.shape
        plane = H * W
    _need(guide, "guide")
    Ry, Rx = len(grid(H, p.patch, p.step)), len(grid(W, p.patch, p.step))
    idx = torch.empty((B, Ry, Rx, p.n2), dtype=torch.int32, device=guide.device)
    n = torch.empty((B, Ry, Rx), dtype=torch.int32, device=guide.device)
    nbytes = int(L.lib().dn_bm3d_match_workspace_bytes(B, H, W, ctypes.byref(p), precision))
    ws, nb = _ws(nbytes, guide.device, None)
    check(L.lib().dn_bm3d_match(_vp(guide), plane, B, H, W, ctypes.byref(p), _sigmas(tau, B), precision, _vp(idx),
                                _vp(n), _vp(ws), nb, _stream(stream)), "dn_bm3d_match")
    return idx, n


def bm3d_match_prethresh(guide: torch.Tensor, tau, thr, p: BM3DPass, stream=None):
    """Block matching on 2D-prethresholded patches (coefficients of magnitude
    <= thr[b] zeroed): guide [B, H, W] (or [B, C, H, W], channel 0).
    Returns (idx int32 [B, Ry, Rx, n2], n int32 [B, Ry, Rx])."""
    if guide.dim() == 4:
        B, C, H, W = guide.shape
        plane = C * H * W
    else:
        B, H, W = guide.shape
        plane = H * W
    _need(guide, "guide")
    Ry, Rx = len(grid(H, p.patch, p.step)), len(grid(W, p.patch, p.step))
    idx = torch.empty((B, Ry, Rx, p.n2), dtype=torch.int32, device=guide.device)
    n = torch.empty((B, Ry, Rx), dtype=torch.int32, device=guide.device)
    check(L.lib().dn_bm3d_match_prethresh(_vp(guide), plane, B, H, W, ctypes.byref(p), _sigmas(tau, B),
                                          _sigmas(thr, B), _vp(idx), _vp(n), _stream(stream)),
          "dn_bm3d_match_prethresh")
    return idx, n


def bm3d_match_cross_terms(guide: torch.Tensor, p: BM3DPass, tau: float, tile_x: int, tile_y: int, stream=None):
    """Raw tensor-core cross terms of one 8 x 16 reference tile (test surface):
    returns (cross [128, nchunks, 128], m, (cy0, cx0)): reference t of the tile
    against candidate (cy0 + 2 c + j // 64, cx0 + j % 64) at cross[t, c, j], the
    dot product of the FP16-rounded patches centred on the tile's constant m."""
    _need(guide, "guide", dim=2)
    H, W = guide.shape
    hs = p.search // 2
    gy, gx = grid(H, 8, p.step), grid(W, 8, p.step)
    y_first, x_first = gy[tile_y * 16], gx[tile_x * 8]
    y_last = gy[min(tile_y * 16 + 15, len(gy) - 1)]
    cy0, cy1 = max(0, y_first - hs), min(H - 8, y_last + hs)
    nchunks = (cy1 - cy0 + 1 + 1) // 2
    buf = torch.zeros(1 + 128 * nchunks * 128, dtype=torch.float32, device=guide.device)
    idx = torch.empty((len(gy), len(gx), p.n2), dtype=torch.int32, device=guide.device)
    n = torch.empty((len(gy), len(gx)), dtype=torch.int32, device=guide.device)
    ws, nb = _ws(int(L.lib().dn_bm3d_match_workspace_bytes(1, H, W, ctypes.byref(p), DN_BF16)), guide.device, None)
    check(L.lib().dn_bm3d_match_cross_terms(_vp(guide), H, W, ctypes.byref(p), float(tau), tile_x, tile_y,
                                            _vp(buf), _vp(idx), _vp(n), _vp(ws), nb, _stream(stream)),
          "dn_bm3d_match_cross_terms")
    return buf[1:].view(128, nchunks, 128), buf[:1], (cy0, max(0, x_first - hs))


def _filter(wiener, img, basic, idx, n, sigma_c, p, precision, stream):
    _need(img, "img", dim=4)
    B, C, H, W = img.shape
    _need(idx, "idx", torch.int32)
    _need(n, "n", torch.int32)
    out = torch.empty_like(img)
    ws, nb = _ws(int(L.lib().dn_bm3d_filter_workspace_bytes(B, C, H, W)), img.device, None)
    sc = farr([float(v) for v in sigma_c])
    if wiener:
        _need(basic, "basic", dim=4)
        st = L.lib().dn_bm3d_filter_wiener(_vp(img), _vp(basic), _vp(idx), _vp(n), B, C, H, W, sc, ctypes.byref(p),
                                           precision, _vp(out), _vp(ws), nb, _stream(stream))
    else:
        st = L.lib().dn_bm3d_filter_hard(_vp(img), _vp(idx), _vp(n), B, C, H, W, sc, ctypes.byref(p), precision,
                                         _vp(out), _vp(ws), nb, _stream(stream))
    check(st, "dn_bm3d_filter_wiener" if wiener else "dn_bm3d_filter_hard")
    return out


def bm3d_filter_hard(img, idx, n, sigma_c: Sequence[float], p: BM3DPass, precision=DN_FP32, stream=None):
    """First-pass filtering + aggregation given match lists; sigma_c is [B*C]."""
    return _filter(False, img, None, idx, n, sigma_c, p, precision, stream)


def bm3d_filter_wiener(noisy, basic, idx, n, sigma_c: Sequence[float], p: BM3DPass, precision=DN_FP32, stream=None):
    """Second-pass filtering + aggregation given match lists on the basic estimate."""
    return _filter(True, noisy, basic, idx, n, sigma_c, p, precision, stream)


def rgb_to_ycc(x: torch.Tensor, stream=None) -> torch.Tensor:
    _need(x, "x", dim=4)
    out = torch.empty_like(x)
    check(L.lib().dn_rgb_to_ycc(_vp(x), _vp(out), x.shape[0], x.shape[2], x.shape[3], _stream(stream)), "dn_rgb_to_ycc")
    return out


def ycc_to_rgb(x: torch.Tensor, stream=None) -> torch.Tensor:
    _need(x, "x", dim=4)
    out = torch.empty_like(x)
    check(L.lib().dn_ycc_to_rgb(_vp(x), _vp(out), x.shape[0], x.shape[2], x.shape[3], _stream(stream)), "dn_ycc_to_rgb")
    return out


def error_reduce(out: torch.Tensor, ref: torch.Tensor, stream=None):
    """Per image FP64 (sum of squared errors of clip(out), max |out - ref|)."""
    _need(out, "out")
    _need(ref, "ref")
    B = out.shape[0]
    sse = torch.empty(B, dtype=torch.float64, device=out.device)
    mx = torch.empty(B, dtype=torch.float64, device=out.device)
    check(L.lib().dn_error_reduce(_vp(out), _vp(ref), B, out[0].numel(), _vp(sse), _vp(mx), _stream(stream)),
          "dn_error_reduce")
    return sse, mx


def conv3x3_fwd(x, w, b=None, relu=False, stream=None):
    _need(x, "x", dim=4)
    _need(w, "w", dim=4)
    N, Cin, H, W = x.shape
    Cout = w.shape[0]
    y = torch.empty((N, Cout, H, W), dtype=torch.float32, device=x.device)
    check(L.lib().dn_conv3x3_fwd(_vp(x), _vp(w), _vp(b), _vp(y), N, Cin, Cout, H, W, int(bool(relu)),
                                 _stream(stream)), "dn_conv3x3_fwd")
    return y


def conv3x3_bwd_data(dy, w, mask=None, stream=None):
    _need(dy, "dy", dim=4)
    _need(w, "w", dim=4)
    N, Cout, H, W = dy.shape
    Cin = w.shape[3]
    dx = torch.empty((N, Cin, H, W), dtype=torch.float32, device=dy.device)
    check(L.lib().dn_conv3x3_bwd_data(_vp(dy), _vp(w), _vp(mask), _vp(dx), N, Cin, Cout, H, W, _stream(stream)),
          "dn_conv3x3_bwd_data")
    return dx


def conv3x3_bwd_weight(x, dy, dw=None, db=None, stream=None):
    """(dw [Cout,3,3,Cin], db [Cout]); writes into dw/db when given (contiguous)."""
    _need(x, "x", dim=4)
    _need(dy, "dy", dim=4)
    N, Cin, H, W = x.shape
    Cout = dy.shape[1]
    dw = torch.empty((Cout, 3, 3, Cin), dtype=torch.float32, device=x.device) if dw is None else dw
    db = torch.empty((Cout,), dtype=torch.float32, device=x.device) if db is None else db
    _need(dw, "dw")
    _need(db, "db")
    if dw.numel() != Cout * 9 * Cin or db.numel() != Cout:
        raise ValueError("dw/db have the wrong size")
    check(L.lib().dn_conv3x3_bwd_weight(_vp(x), _vp(dy), _vp(dw), _vp(db), N, Cin, Cout, H, W, _stream(stream)),
          "dn_conv3x3_bwd_weight")
    return dw, db


def cnn_forward(noisy, pre, weights, layers=10, width=32, precision=DN_FP32, stream=None):
    """Residual network pre + 255 F([pre, noisy] / 255) on planes [N, H, W]
    (grey network) or [N, 3, H, W] (colour-native network)."""
    colour = noisy.dim() == 4
    _need(noisy, "noisy", dim=4 if colour else 3)
    _need(pre, "pre", dim=4 if colour else 3)
    if colour and noisy.shape[1] != 3:
        raise ValueError("a colour-native network takes 3 planes")
    N, H, W = noisy.shape[0], noisy.shape[-2], noisy.shape[-1]
    cnn = make_cnn(weights, layers, width, precision, 3 if colour else 1)
    out = torch.empty_like(noisy)
    ws, nb = _ws(int(L.lib().dn_cnn_workspace_bytes(N, H, W, ctypes.byref(cnn))), noisy.device, None)
    check(L.lib().dn_cnn_forward(_vp(noisy), _vp(pre), _vp(out), N, H, W, ctypes.byref(cnn), _vp(ws), nb,
                                 _stream(stream)), "dn_cnn_forward")
    return out


def cnn_grad(noisy, pre, clean, weights, layers=10, width=32, grad=None, loss=None, workspace=None, stream=None):
    """Gradient of the L1 loss of Eq. 2 for the grey network on planes
    [N, H, W] with the BF16 tensor-core forward and backward kernels.
    Returns (grad in the layout of weights, loss_sum device double [1])."""
    _need(noisy, "noisy", dim=3)
    _need(pre, "pre", dim=3)
    _need(clean, "clean", dim=3)
    N, H, W = noisy.shape
    cnn = make_cnn(weights, layers, width, DN_BF16, 1)
    grad = torch.empty_like(weights) if grad is None else grad
    if loss is None:
        loss = torch.zeros(1, dtype=torch.float64, device=noisy.device)
    ws, nb = _ws(int(L.lib().dn_cnn_grad_workspace_bytes(N, H, W, ctypes.byref(cnn))), noisy.device, workspace)
    check(L.lib().dn_cnn_grad(_vp(noisy), _vp(pre), _vp(clean), N, H, W, ctypes.byref(cnn), _vp(grad), _vp(loss),
                              _vp(ws), nb, _stream(stream)), "dn_cnn_grad")
    return grad, loss


def conv3x3_tc_pair_fwd(x_nhwc, wa, ba, wb, bb, stream=None):
    """Two hidden 32 -> 32 layers (bias + ReLU each) in one tensor-core pass."""
    _need(x_nhwc, "x_nhwc", torch.bfloat16, dim=4)
    N, H, W, C = x_nhwc.shape
    y = torch.empty_like(x_nhwc)
    ws, nb = _ws(2 * 9 * C * C * 2, x_nhwc.device, None)
    check(L.lib().dn_conv3x3_tc_pair_fwd(_vp(x_nhwc), _vp(wa.contiguous()), _vp(ba.contiguous()),
                                         _vp(wb.contiguous()), _vp(bb.contiguous()), _vp(y), N, H, W, C, _vp(ws), nb,
                                         _stream(stream)), "dn_conv3x3_tc_pair_fwd")
    return y


def conv3x3_tc_bwd_weight(x_nhwc, g_nhwc, stream=None):
    """(dw [C, 3, 3, C], db [C]) of one hidden tensor-core layer (C = 32)."""
    _need(x_nhwc, "x_nhwc", torch.bfloat16, dim=4)
    _need(g_nhwc, "g_nhwc", torch.bfloat16, dim=4)
    N, H, W, C = x_nhwc.shape
    dw = torch.empty((C, 3, 3, C), dtype=torch.float32, device=x_nhwc.device)
    db = torch.empty(C, dtype=torch.float32, device=x_nhwc.device)
    ws, nb = _ws(int(L.lib().dn_conv3x3_tc_bwd_workspace_bytes(N, H, W, C)), x_nhwc.device, None)
    check(L.lib().dn_conv3x3_tc_bwd_weight(_vp(x_nhwc), _vp(g_nhwc), _vp(dw), _vp(db), N, H, W, C, _vp(ws), nb,
                                           _stream(stream)), "dn_conv3x3_tc_bwd_weight")
    return dw, db


def conv3x3_tc_bwd_data(g_nhwc, w, mask_nhwc=None, stream=None):
    """Data gradient (NHWC bf16) of one hidden tensor-core layer with weights
    w [C, 3, 3, C], zeroed where mask_nhwc (the layer input) is not positive."""
    _need(g_nhwc, "g_nhwc", torch.bfloat16, dim=4)
    N, H, W, C = g_nhwc.shape
    dx = torch.empty_like(g_nhwc)
    ws, nb = _ws(int(L.lib().dn_conv3x3_tc_bwd_workspace_bytes(N, H, W, 32)) if C == 32 else 9 * C * C * 2,
                 g_nhwc.device, None)
    check(L.lib().dn_conv3x3_tc_bwd_data(_vp(g_nhwc), _vp(w.contiguous()), _vp(mask_nhwc) if mask_nhwc is not None
                                         else None, _vp(dx), N, H, W, C, _vp(ws), nb, _stream(stream)),
          "dn_conv3x3_tc_bwd_data")
    return dx


def conv3x3_tc_fwd(x_nhwc, w, b, relu=True, stream=None):
    """One C -> C layer on the tensor cores (C = 32 or 64): x_nhwc bf16 [N, H, W, C] -> same."""
    _need(x_nhwc, "x_nhwc", torch.bfloat16, dim=4)
    _need(w, "w", dim=4)
    _need(b, "b", dim=1)
    N, H, W, C = x_nhwc.shape
    if C not in (32, 64) or tuple(w.shape) != (C, 3, 3, C) or b.numel() != C:
        raise ValueError("conv3x3_tc_fwd handles C -> C channels, C = 32 or 64")
    y = torch.empty_like(x_nhwc)
    ws = torch.empty(9 * C * C * 2, dtype=torch.uint8, device=x_nhwc.device)
    check(L.lib().dn_conv3x3_tc_fwd(_vp(x_nhwc), _vp(w), _vp(b), _vp(y), N, H, W, C, int(bool(relu)), _vp(ws),
                                    ws.numel(), _stream(stream)), "dn_conv3x3_tc_fwd")
    return y


def device_error(reset: bool = True) -> int:
    """The library's device error word (nonzero: a bounded wait ran out)."""
    code = ctypes.c_int(0)
    check(L.lib().dn_device_error(ctypes.byref(code), int(reset)), "dn_device_error")
    return code.value


def cnn_pack_input(pre, noisy, stream=None):
    """z [N, 2, H, W] = [pre / 255, noisy / 255] (Eq. 3) from planes [N, H, W]."""
    _need(pre, "pre", dim=3)
    _need(noisy, "noisy", dim=3)
    N, H, W = pre.shape
    z = torch.empty((N, 2, H, W), dtype=torch.float32, device=pre.device)
    check(L.lib().dn_cnn_pack_input(_vp(pre), _vp(noisy), _vp(z), N, H, W, _stream(stream)), "dn_cnn_pack_input")
    return z


def cnn_residual_out(pre, r, out=None, stream=None):
    """out = pre + 255 r (Eq. 2); out may be given (same shape as pre)."""
    _need(pre, "pre")
    _need(r, "r")
    out = torch.empty_like(pre) if out is None else out
    _need(out, "out")
    if out.numel() != pre.numel() or r.numel() != pre.numel():
        raise ValueError("pre, r and out must have the same number of elements")
    check(L.lib().dn_cnn_residual_out(_vp(pre), _vp(r), _vp(out), pre.numel(), _stream(stream)), "dn_cnn_residual_out")
    return out


def relu_bwd(g, y, stream=None):
    _need(g, "g")
    _need(y, "y")
    out = torch.empty_like(g)
    check(L.lib().dn_relu_bwd(_vp(g), _vp(y), _vp(out), g.numel(), _stream(stream)), "dn_relu_bwd")
    return out


def l1_residual_grad(r, pre, clean, loss_sum=None, stream=None):
    _need(r, "r")
    dr = torch.empty_like(r)
    check(L.lib().dn_l1_residual_grad(_vp(r), _vp(pre), _vp(clean), _vp(dr), r.numel(), _vp(loss_sum),
                                      _stream(stream)), "dn_l1_residual_grad")
    return dr


def adam_step(param, grad, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    for name, x in (("param", param), ("grad", grad), ("m", m), ("v", v)):
        _need(x, name)
    check(L.lib().dn_adam_step(_vp(param), _vp(grad), _vp(m), _vp(v), param.numel(), int(t), lr, beta1, beta2, eps,
                               _stream(stream)), "dn_adam_step")


# ---- layers of the flexible lightweight network (Sec. III) -------------------

def dw3x3_fwd(x, w, b=None, stride=1, relu=False, stream=None):
    """Depthwise 3x3 (zero padding 1, stride 1 or 2): x [N, C, H, W], w [C, 3, 3], b [C]."""
    _need(x, "x", dim=4)
    _need(w, "w")
    N, C, H, W = x.shape
    y = torch.empty(N, C, (H + stride - 1) // stride, (W + stride - 1) // stride, device=x.device)
    check(L.lib().dn_dw3x3_fwd(_vp(x), _vp(w), _vp(b), _vp(y), N, C, H, W, stride, int(relu), _stream(stream)),
          "dn_dw3x3_fwd")
    return y


def dw3x3_bwd(x, g, w, stride=1, need_dx=True, stream=None):
    """(dx or None, dw [C, 3, 3], db [C]) of the depthwise layer for g = dL/dy."""
    _need(x, "x", dim=4)
    _need(g, "g", dim=4)
    N, C, H, W = x.shape
    dx = torch.empty_like(x) if need_dx else None
    dw = torch.empty(C, 3, 3, device=x.device)
    db = torch.empty(C, device=x.device)
    check(L.lib().dn_dw3x3_bwd(_vp(x), _vp(g), _vp(w), _vp(dx), _vp(dw), _vp(db), N, C, H, W, stride,
                               _stream(stream)), "dn_dw3x3_bwd")
    return dx, dw, db


def pw_fwd(x, w, b=None, relu=False, transposed=False, precision=DN_FP32, stream=None):
    """Pointwise: x [N, Cin, H, W], w [Cout, Cin] -> [N, Cout, H, W]; transposed: w [Cin', Cout'] used as W^T.
    precision DN_BF16: the tensor-core kernel (BF16 operands, FP32 accumulation)."""
    _need(x, "x", dim=4)
    _need(w, "w")
    N, Cin, H, W = x.shape
    Cout = w.shape[1] if transposed else w.shape[0]
    y = torch.empty(N, Cout, H, W, device=x.device)
    fn = L.lib().dn_pw_fwd_bf16 if precision == DN_BF16 else L.lib().dn_pw_fwd
    check(fn(_vp(x), _vp(w), _vp(b), _vp(y), N, Cin, Cout, H * W, int(relu), int(transposed), _stream(stream)),
          "dn_pw_fwd")
    return y


def pw_bwd_weight(x, g, stream=None):
    """(dw [Cout, Cin], db [Cout]) of a pointwise layer."""
    _need(x, "x", dim=4)
    _need(g, "g", dim=4)
    N, Cin, H, W = x.shape
    Cout = g.shape[1]
    dw = torch.empty(Cout, Cin, device=x.device)
    db = torch.empty(Cout, device=x.device)
    check(L.lib().dn_pw_bwd_weight(_vp(x), _vp(g), _vp(dw), _vp(db), N, Cin, Cout, H * W, _stream(stream)),
          "dn_pw_bwd_weight")
    return dw, db


def deconv2x2_fwd(x, w, b=None, skip=None, precision=DN_FP32, stream=None):
    """Transposed 2x2 conv, stride 2: x [N, Cin, H, W], w [Cin, Cout, 2, 2] -> [N, Cout, 2H, 2W] (+ skip).
    precision DN_BF16: four tensor-core GEMMs, one per tap."""
    _need(x, "x", dim=4)
    _need(w, "w")
    N, Cin, H, W = x.shape
    Cout = w.shape[1]
    y = torch.empty(N, Cout, 2 * H, 2 * W, device=x.device)
    fn = L.lib().dn_deconv2x2_fwd_bf16 if precision == DN_BF16 else L.lib().dn_deconv2x2_fwd
    check(fn(_vp(x), _vp(w), _vp(b), _vp(skip), _vp(y), N, Cin, Cout, H, W, _stream(stream)), "dn_deconv2x2_fwd")
    return y


def deconv2x2_bwd(x, g, w, need_dx=True, stream=None):
    """(dx or None, dw [Cin, Cout, 2, 2], db [Cout]) of the transposed convolution."""
    _need(x, "x", dim=4)
    _need(g, "g", dim=4)
    N, Cin, H, W = x.shape
    Cout = w.shape[1]
    dx = torch.empty_like(x) if need_dx else None
    dw = torch.empty(Cin, Cout, 2, 2, device=x.device)
    db = torch.empty(Cout, device=x.device)
    check(L.lib().dn_deconv2x2_bwd(_vp(x), _vp(g), _vp(w), _vp(dx), _vp(dw), _vp(db), N, Cin, Cout, H, W,
                                   _stream(stream)), "dn_deconv2x2_bwd")
    return dx, dw, db


def fl_pack_input(pre, noisy, sigma, stream=None):
    """z [N, 3, H, W] = [pre / 255, noisy / 255, sigma_n / 255] from planes [N, H, W]."""
    _need(pre, "pre", dim=3)
    _need(noisy, "noisy", dim=3)
    N, H, W = pre.shape
    z = torch.empty(N, 3, H, W, device=pre.device)
    check(L.lib().dn_fl_pack_input(_vp(pre), _vp(noisy), _sigmas(sigma, N), _vp(z), N, H, W, _stream(stream)),
          "dn_fl_pack_input")
    return z


class profile:
    """Context manager timing every library kernel with CUDA events on its stream.

    Usage: with profile() as prof: ...; prof.result -> {name: (launches, ms)}."""

    def __enter__(self):
        L.lib().dn_profile_reset()
        L.lib().dn_profile_enable(1)
        self.result = {}
        return self

    def __exit__(self, *exc):
        L.lib().dn_profile_enable(0)
        self.result = read_profile()
        L.lib().dn_profile_reset()
        return False


def read_profile():
    n = L.lib().dn_profile_read(None, 0, 0, None, None)
    if n <= 0:
        return {}
    stride = 64
    names = ctypes.create_string_buffer(stride * n)
    launches = (ctypes.c_int * n)()
    ms = (ctypes.c_double * n)()
    L.lib().dn_profile_read(names, stride, n, launches, ms)
    out = {}
    for k in range(n):
        nm = names.raw[k * stride:(k + 1) * stride].split(b"\0", 1)[0].decode()
        out[nm] = (launches[k], ms[k])
    return out

"""Thin ctypes binding of libdenoise.so (include/denoise.h).

Argument marshalling only: every computation runs in the library's CUDA
kernels.  Tensors are torch CUDA tensors (PyTorch provides device memory and
streams); their data pointers and the current stream are handed to the C ABI.
If the library is missing this module raises: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdenoise.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "denoise.h")

DN_OK, DN_EINVAL, DN_ENOMEM, DN_ECUDA, DN_EDEVICE, DN_EUNSUPPORTED = 0, -1, -2, -3, -4, -5
DN_FP32, DN_BF16, DN_BF16_MATCH = 0, 1, 2
DN_PREFILTER_BM3D, DN_PREFILTER_NLM = 0, 1


class DenoiseError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__("%s failed: %s (%d)" % (what, strerror(status), status))


class BM3DPass(ctypes.Structure):
    _fields_ = [("patch", ctypes.c_int), ("step", ctypes.c_int), ("search", ctypes.c_int), ("n2", ctypes.c_int),
                ("tau", ctypes.c_float), ("tau_high", ctypes.c_float), ("lambda3d", ctypes.c_float),
                ("beta", ctypes.c_float), ("lambda2d", ctypes.c_float), ("patch_high", ctypes.c_int),
                ("step_high", ctypes.c_int)]


class BM3DParams(ctypes.Structure):
    _fields_ = [("hard", BM3DPass), ("wiener", BM3DPass), ("precision", ctypes.c_int),
                ("sigma_regime", ctypes.c_int)]


class NLMParams(ctypes.Structure):
    _fields_ = [("patch", ctypes.c_int), ("search", ctypes.c_int), ("h_over_sigma", ctypes.c_float)]


class CNN(ctypes.Structure):
    _fields_ = [("layers", ctypes.c_int), ("width", ctypes.c_int), ("weights", ctypes.c_void_p),
                ("precision", ctypes.c_int), ("channels", ctypes.c_int)]


_lib = None


def lib():
    """Loads libdenoise.so (built by paper_2403_03488_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libdenoise.so is not built (run __graft_entry__.build()); no fallback exists")
    L = ctypes.CDLL(LIB_PATH)
    vp, sz, i, f, d = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_float, ctypes.c_double
    fp = ctypes.POINTER(ctypes.c_float)
    ip = ctypes.POINTER(ctypes.c_int)
    dp = ctypes.POINTER(ctypes.c_double)
    P = ctypes.POINTER
    sig = {
        "dn_bm3d_default_params": (None, [P(BM3DParams)]),
        "dn_bm3d_high_noise_params": (None, [P(BM3DParams)]),
        "dn_nlm_default_params": (None, [P(NLMParams)]),
        "dn_cnn_param_count": (sz, [i, i]),
        "dn_cnn_param_count_c": (sz, [i, i, i]),
        "dn_bm3d_grid": (i, [i, i, i, ip]),
        "dn_bm3d_workspace_bytes": (sz, [i, i, i, i, P(BM3DParams)]),
        "dn_nlm_workspace_bytes": (sz, [i, i, i, i, P(NLMParams)]),
        "dn_hybrid_workspace_bytes": (sz, [i, i, i, i, i, vp, P(CNN)]),
        "denoise_bm3d": (i, [vp, vp, i, i, i, i, fp, P(BM3DParams), vp, sz, vp]),
        "denoise_nlm": (i, [vp, vp, i, i, i, i, fp, P(NLMParams), vp, sz, vp]),
        "denoise_hybrid": (i, [vp, vp, i, i, i, i, fp, i, vp, P(CNN), vp, sz, vp]),
        "dn_strerror": (ctypes.c_char_p, [i]),
        "denoise_bm3d_noalloc": (i, [vp, vp, i, i, i, i, fp, P(BM3DParams), vp]),
        "dn_noalloc_scratch_bytes": (sz, []),
        "dn_bm3d_halo": (i, [P(BM3DParams)]),
        "dn_bm3d_tiled_workspace_bytes": (sz, [i, i, i, P(BM3DParams), i, i]),
        "denoise_bm3d_tiled": (i, [vp, vp, i, i, i, f, P(BM3DParams), i, i, vp, sz, vp]),
        "dn_bm3d_match": (i, [vp, sz, i, i, i, P(BM3DPass), fp, i, vp, vp, vp, sz, vp]),
        "dn_bm3d_match_workspace_bytes": (sz, [i, i, i, P(BM3DPass), i]),
        "dn_bm3d_match_prethresh": (i, [vp, sz, i, i, i, P(BM3DPass), fp, fp, vp, vp, vp]),
        "dn_bm3d_match_cross_terms": (i, [vp, i, i, P(BM3DPass), f, i, i, vp, vp, vp, vp, sz, vp]),
        "dn_bm3d_filter_hard": (i, [vp, vp, vp, i, i, i, i, fp, P(BM3DPass), i, vp, vp, sz, vp]),
        "dn_bm3d_filter_wiener": (i, [vp, vp, vp, vp, i, i, i, i, fp, P(BM3DPass), i, vp, vp, sz, vp]),
        "dn_bm3d_filter_workspace_bytes": (sz, [i, i, i, i]),
        "dn_rgb_to_ycc": (i, [vp, vp, i, i, i, vp]),
        "dn_ycc_to_rgb": (i, [vp, vp, i, i, i, vp]),
        "dn_error_reduce": (i, [vp, vp, i, sz, vp, vp, vp]),
        "dn_conv3x3_fwd": (i, [vp, vp, vp, vp, i, i, i, i, i, i, vp]),
        "dn_conv3x3_bwd_data": (i, [vp, vp, vp, vp, i, i, i, i, i, vp]),
        "dn_conv3x3_bwd_weight": (i, [vp, vp, vp, vp, i, i, i, i, i, vp]),
        "dn_cnn_forward": (i, [vp, vp, vp, i, i, i, P(CNN), vp, sz, vp]),
        "dn_cnn_workspace_bytes": (sz, [i, i, i, P(CNN)]),
        "dn_cnn_grad": (i, [vp, vp, vp, i, i, i, P(CNN), vp, vp, vp, sz, vp]),
        "dn_cnn_grad_workspace_bytes": (sz, [i, i, i, P(CNN)]),
        "dn_conv3x3_tc_bwd_workspace_bytes": (sz, [i, i, i, i]),
        "dn_pw_fwd_bf16": (i, [vp, vp, vp, vp, i, i, i, i, i, i, vp]),
        "dn_deconv2x2_fwd_bf16": (i, [vp, vp, vp, vp, vp, i, i, i, i, i, vp]),
        "dn_conv3x3_tc_pair_fwd": (i, [vp, vp, vp, vp, vp, vp, i, i, i, i, vp, sz, vp]),
        "dn_conv3x3_tc_bwd_weight": (i, [vp, vp, vp, vp, i, i, i, i, vp, sz, vp]),
        "dn_conv3x3_tc_bwd_data": (i, [vp, vp, vp, vp, i, i, i, i, vp, sz, vp]),
        "dn_conv3x3_tc_fwd": (i, [vp, vp, vp, vp, i, i, i, i, i, vp, sz, vp]),
        "dn_device_error": (i, [ip, i]),
        "dn_cnn_pack_input": (i, [vp, vp, vp, i, i, i, vp]),
        "dn_cnn_residual_out": (i, [vp, vp, vp, sz, vp]),
        "dn_relu_bwd": (i, [vp, vp, vp, sz, vp]),
        "dn_l1_residual_grad": (i, [vp, vp, vp, vp, sz, vp, vp]),
        "dn_adam_step": (i, [vp, vp, vp, vp, sz, i, f, f, f, f, vp]),
        "dn_profile_enable": (None, [i]),
        "dn_profile_read": (i, [ctypes.c_char_p, i, i, ip, dp]),
        "dn_profile_reset": (None, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def header_functions(path: str = HEADER):
    """Names of every function declared in include/denoise.h."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b([A-Za-z_][A-Za-z0-9_]*)\s*\(", text)
    skip = {"if", "while", "for", "sizeof", "return", "defined"}
    decl = set()
    for m in re.finditer(r"^[A-Za-z_][A-Za-z0-9_ \*]*?\b([A-Za-z_][A-Za-z0-9_]*)\s*\(", text, flags=re.M):
        if m.group(1) not in skip and not text[m.start():m.start() + 8].startswith("typedef"):
            decl.add(m.group(1))
    return sorted(n for n in decl if n in names)


def strerror(status: int) -> str:
    try:
        return lib().dn_strerror(int(status)).decode()
    except Exception:
        return "status %d" % status


def check(status: int, what: str):
    if status != DN_OK:
        raise DenoiseError(status, what)


def default_bm3d_params(precision: int = DN_FP32, regime: int = 0, high_noise_patches: bool = False) -> BM3DParams:
    """The library defaults; high_noise_patches: the larger patches of BM3D's
    high-noise profile above sigma 40 (12 x 12 step 4, 11 x 11 step 6)."""
    p = BM3DParams()
    if high_noise_patches:
        lib().dn_bm3d_high_noise_params(ctypes.byref(p))
    else:
        lib().dn_bm3d_default_params(ctypes.byref(p))
    p.precision = precision
    p.sigma_regime = regime
    return p


def default_nlm_params() -> NLMParams:
    p = NLMParams()
    lib().dn_nlm_default_params(ctypes.byref(p))
    return p


def farr(values):
    vals = [float(v) for v in values]
    return (ctypes.c_float * len(vals))(*vals)

"""The C-ABI library loads without a GPU, exports every function declared in
include/denoise.h, and rejects bad arguments on the host before any launch."""
import ctypes

import pytest

from paper_2403_03488_gb300 import build as B
from paper_2403_03488_gb300 import _lib as L


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.lib()


def test_exports_every_declared_function(lib):
    names = L.header_functions()
    assert len(names) >= 29
    raw = ctypes.CDLL(L.LIB_PATH)
    missing = [n for n in names if not hasattr(raw, n)]
    assert not missing, missing
    for core in ("denoise_bm3d", "denoise_nlm", "denoise_hybrid", "dn_strerror"):
        assert core in names


def test_param_count_and_defaults(lib):
    assert lib.dn_cnn_param_count(10, 32) == 2 * 32 * 9 + 32 + 8 * (32 * 32 * 9 + 32) + 32 * 9 + 1
    assert lib.dn_cnn_param_count_c(10, 32, 1) == lib.dn_cnn_param_count(10, 32)
    # colour-native: 6 -> 64 -> ... -> 64 -> 3
    assert lib.dn_cnn_param_count_c(16, 64, 3) == 6 * 64 * 9 + 64 + 14 * (64 * 64 * 9 + 64) + 3 * 64 * 9 + 3
    assert lib.dn_cnn_param_count_c(10, 32, 2) == 0
    p = L.default_bm3d_params()
    assert (p.hard.patch, p.hard.step, p.hard.search, p.hard.n2) == (8, 3, 39, 16)
    assert (p.hard.tau, p.hard.tau_high, p.hard.lambda3d, p.hard.beta) == (2500.0, 5000.0, 2.700000047683716, 2.0)
    assert (p.wiener.n2, p.wiener.tau, p.wiener.tau_high) == (32, 400.0, 3500.0)
    assert (p.hard.lambda2d, p.wiener.lambda2d) == (2.0, 0.0)
    q = L.default_nlm_params()
    assert (q.patch, q.search) == (7, 21) and abs(q.h_over_sigma - 0.4) < 1e-7


def test_grid_matches_oracle(lib, oracle):
    from paper_2403_03488_gb300 import api
    for n in (8, 9, 11, 37, 128, 129, 512, 1024, 1600):
        assert api.grid(n) == list(oracle.grid(n))
    assert api.grid(7) == []


def _call_bm3d(lib, B=1, C=1, H=32, W=32, sigma=25.0, p=None, ws_bytes=1 << 30, ws=1):
    p = p or L.default_bm3d_params()
    sig = L.farr([sigma] * max(B, 1))
    return lib.denoise_bm3d(ctypes.c_void_p(16), ctypes.c_void_p(32), B, C, H, W, sig, ctypes.byref(p),
                            ctypes.c_void_p(ws) if ws else None, ws_bytes, None)


def test_bm3d_rejects_bad_arguments_on_host(lib):
    assert _call_bm3d(lib, B=0) == L.DN_EINVAL
    assert _call_bm3d(lib, C=2) == L.DN_EINVAL
    assert _call_bm3d(lib, H=7) == L.DN_EINVAL
    assert _call_bm3d(lib, sigma=0.0) == L.DN_EINVAL
    assert _call_bm3d(lib, sigma=float("nan")) == L.DN_EINVAL
    p = L.default_bm3d_params()
    p.hard.n2 = 12
    assert _call_bm3d(lib, p=p) == L.DN_EINVAL
    p = L.default_bm3d_params()
    p.wiener.search = 38
    assert _call_bm3d(lib, p=p) == L.DN_EINVAL
    p = L.default_bm3d_params()
    p.hard.patch = 7
    assert _call_bm3d(lib, p=p) == L.DN_EINVAL
    p = L.default_bm3d_params()
    p.hard.lambda2d = -1.0
    assert _call_bm3d(lib, p=p) == L.DN_EINVAL
    p.hard.lambda2d = float("inf")
    assert _call_bm3d(lib, p=p) == L.DN_EINVAL
    # the prethresholded matcher checks its host arrays before any launch
    q = L.default_bm3d_params().hard
    dummy = ctypes.c_void_p(16)
    for tau, thr in (([5000.0], [-1.0]), ([5000.0], [float("nan")]), ([0.0], [100.0])):
        assert lib.dn_bm3d_match_prethresh(dummy, 32 * 32, 1, 32, 32, ctypes.byref(q), L.farr(tau), L.farr(thr),
                                           dummy, dummy, None) == L.DN_EINVAL
    assert lib.dn_bm3d_match_prethresh(dummy, 32 * 32, 1, 32, 32, ctypes.byref(q), L.farr([5000.0]), None,
                                       dummy, dummy, None) == L.DN_EINVAL
    assert _call_bm3d(lib, ws=0) == L.DN_ENOMEM
    assert _call_bm3d(lib, ws_bytes=100) == L.DN_ENOMEM
    assert lib.denoise_bm3d(None, None, 1, 1, 32, 32, L.farr([25.0]), ctypes.byref(L.default_bm3d_params()),
                            None, 0, None) == L.DN_EINVAL


def test_workspace_queries(lib):
    p = L.default_bm3d_params()
    a = lib.dn_bm3d_workspace_bytes(1, 1, 64, 64, ctypes.byref(p))
    b = lib.dn_bm3d_workspace_bytes(2, 1, 64, 64, ctypes.byref(p))
    c = lib.dn_bm3d_workspace_bytes(1, 3, 64, 64, ctypes.byref(p))
    assert 0 < a < b and a < c
    assert lib.dn_bm3d_workspace_bytes(1, 1, 4, 64, ctypes.byref(p)) == 0
    assert lib.dn_nlm_workspace_bytes(1, 1, 64, 64, None) == 0
    assert lib.dn_nlm_workspace_bytes(1, 3, 64, 64, None) > 0


def test_nlm_and_hybrid_reject_bad_arguments(lib):
    q = L.default_nlm_params()
    q.patch = 6
    sig = L.farr([25.0])
    assert lib.denoise_nlm(ctypes.c_void_p(16), ctypes.c_void_p(32), 1, 1, 32, 32, sig, ctypes.byref(q), None, 0,
                           None) == L.DN_EINVAL
    q = L.default_nlm_params()
    assert lib.denoise_nlm(ctypes.c_void_p(16), ctypes.c_void_p(32), 1, 1, 3, 32, sig, ctypes.byref(q), None, 0,
                           None) == L.DN_EINVAL
    cnn = L.CNN(1, 32, ctypes.c_void_p(64), 0)
    p = L.default_bm3d_params()
    assert lib.denoise_hybrid(ctypes.c_void_p(16), ctypes.c_void_p(32), 1, 1, 32, 32, sig, 0,
                              ctypes.cast(ctypes.byref(p), ctypes.c_void_p), ctypes.byref(cnn), None, 0,
                              None) == L.DN_EINVAL
    cnn = L.CNN(10, 32, ctypes.c_void_p(64), 0)
    assert lib.denoise_hybrid(ctypes.c_void_p(16), ctypes.c_void_p(32), 1, 1, 32, 32, sig, 7,
                              ctypes.cast(ctypes.byref(p), ctypes.c_void_p), ctypes.byref(cnn), None, 0,
                              None) == L.DN_EINVAL
    assert lib.denoise_hybrid(ctypes.c_void_p(16), ctypes.c_void_p(32), 1, 1, 32, 32, sig, 0,
                              ctypes.cast(ctypes.byref(p), ctypes.c_void_p), ctypes.byref(cnn), None, 0,
                              None) == L.DN_ENOMEM


def test_layer_entry_points_reject_bad_arguments(lib):
    v = ctypes.c_void_p(64)
    assert lib.dn_conv3x3_fwd(v, v, None, v, 1, 0, 32, 8, 8, 1, None) == L.DN_EINVAL
    assert lib.dn_conv3x3_fwd(v, v, None, v, 1, 65, 32, 8, 8, 1, None) == L.DN_EINVAL
    assert lib.dn_conv3x3_bwd_data(v, None, None, v, 1, 2, 32, 8, 8, None) == L.DN_EINVAL
    assert lib.dn_adam_step(v, v, v, v, 10, 0, 1e-3, 0.9, 0.999, 1e-8, None) == L.DN_EINVAL
    assert lib.dn_l1_residual_grad(v, v, v, v, 0, None, None) == L.DN_EINVAL
    assert lib.dn_error_reduce(v, v, 0, 10, v, v, None) == L.DN_EINVAL
    bp = L.default_bm3d_params().hard
    assert lib.dn_bm3d_match(v, 64, 1, 8, 8, ctypes.byref(bp), L.farr([0.0]), 0, v, v, None, 0, None) == L.DN_EINVAL
    assert lib.dn_bm3d_match(v, 10, 1, 8, 8, ctypes.byref(bp), L.farr([1.0]), 0, v, v, None, 0, None) == L.DN_EINVAL
    assert lib.dn_bm3d_filter_hard(v, v, v, 1, 1, 8, 8, L.farr([1.0]), ctypes.byref(bp), 0, v, None, 0,
                                   None) == L.DN_ENOMEM
    assert lib.dn_bm3d_filter_hard(v, v, v, 1, 1, 8, 8, L.farr([-1.0]), ctypes.byref(bp), 0, v, v, 1 << 20,
                                   None) == L.DN_EINVAL


def test_strerror(lib):
    for s in (0, -1, -2, -3, -4, -5):
        assert lib.dn_strerror(s)
    assert b"workspace" in lib.dn_strerror(L.DN_ENOMEM)


def test_noalloc_scratch_size_matches_header(lib):
    """The size the library reports for its fixed no-allocation array is the
    one include/denoise.h defines (read from the header text)."""
    import os
    import re
    hdr = open(os.path.join(os.path.dirname(L.LIB_PATH), "..", "include", "denoise.h")).read()
    m = re.search(r"#define\s+DN_NOALLOC_SCRATCH_BYTES\s+\((\d+)u\s*<<\s*(\d+)\)", hdr)
    assert m, "DN_NOALLOC_SCRATCH_BYTES not found in the header"
    assert lib.dn_noalloc_scratch_bytes() == int(m.group(1)) << int(m.group(2))


def test_high_noise_first_pass_window_limit_is_checked_before_launch(lib):
    """A sigma > 40 image whose prethresholded first pass would stage more than
    200 KB of window (step 12, search 21, 512 wide) is refused with
    DN_EUNSUPPORTED on the host.  With sigma_regime 1 or lambda2d = 0 the first
    pass matches raw pixels, so only the workspace check remains (a 0-byte
    workspace fails it)."""
    p = L.default_bm3d_params()
    p.hard.step = 12
    p.hard.search = 21
    assert _call_bm3d(lib, H=64, W=512, sigma=50.0, p=p) == L.DN_EUNSUPPORTED
    p.sigma_regime = 1
    p2 = L.default_bm3d_params()
    p2.hard.step, p2.hard.search = 12, 21
    p2.hard.lambda2d = 0.0
    assert _call_bm3d(lib, H=64, W=512, sigma=50.0, p=p, ws_bytes=0) == L.DN_ENOMEM
    assert _call_bm3d(lib, H=64, W=512, sigma=50.0, p=p2, ws_bytes=0) == L.DN_ENOMEM

"""denoise_bm3d_noalloc: BM3D for callers that may not allocate device memory
(a plug-in inside an application that owns the device-memory budget, or a
latency-critical loop that cannot risk an allocation that blocks on the
device).  Its workspace is a fixed device array inside the library.

Two calls in a row through the C ABI, on different shapes and noise levels,
must each equal denoise_bm3d (caller-provided workspace) bit for bit: BM3D
here sums its aggregation terms exactly in fixed point, so the result does not
depend on where the workspace lives or what it held before.  A request that
needs more than the fixed array is refused on the host.  This file is collected last so that a
run stopping at its first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

from gpu_util import dev, host, need_gpu
from paper_2403_03488_gb300 import synth

pytestmark = pytest.mark.gpu

def test_noalloc_matches_denoise_bm3d_on_two_calls_in_a_row():
    need_gpu()
    import torch
    from paper_2403_03488_gb300 import api
    from paper_2403_03488_gb300 import _lib as L

    cases = [(1, 96, 112, [25.0, 50.0]), (3, 80, 72, [15.0])]
    for C, H, W, sigmas in cases:
        B = len(sigmas)
        _, noisy = synth.make_batch(range(200, 200 + B), H, W, sigmas, C=C)
        x = dev(noisy)
        p = api.default_bm3d_params()
        out = torch.full_like(x, float("nan"))
        st = L.lib().denoise_bm3d_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), B, C, H, W,
                                          L.farr(sigmas), ctypes.byref(p),
                                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == L.DN_OK, L.strerror(st)
        ref = host(api.denoise_bm3d(x, sigmas, p))
        got = host(out)
        assert np.isfinite(got).all()
        np.testing.assert_array_equal(got, ref)


def test_noalloc_refuses_requests_beyond_the_fixed_array():
    need_gpu()
    from paper_2403_03488_gb300 import api
    from paper_2403_03488_gb300 import _lib as L
    p = api.default_bm3d_params()
    cap = api.noalloc_scratch_bytes()
    assert api.bm3d_workspace_bytes(1, 1, 512, 512, p) <= cap
    assert api.bm3d_workspace_bytes(1, 3, 512, 512, p) > cap
    x = dev(np.zeros((1, 3, 512, 512), np.float32))
    with pytest.raises(L.DenoiseError) as e:
        api.denoise_bm3d_noalloc(x, 25.0, p)
    assert e.value.status == L.DN_ENOMEM

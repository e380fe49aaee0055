"""Shared helpers of the GPU parity tests (no method arithmetic here)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2403_03488_gb300 import build
    build.build()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def footprint(idx_list, n, W, shape):
    """Pixels covered by the first n patches (8x8) of each list."""
    m = np.zeros(shape, bool)
    for lst, k in zip(idx_list, n):
        for p in lst[:k]:
            y, x = divmod(int(p), W)
            m[y:y + 8, x:x + 8] = True
    return m

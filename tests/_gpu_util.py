"""Helpers shared by the GPU tests: build/load the library, move data, compare."""
import numpy as np
import pytest


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2312_00538_gb300 as ab
    return torch, ab


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def to_dev(torch, a, dtype):
    """Column-major n x nrhs host array -> contiguous device tensor of shape (nrhs, n)."""
    a = np.asarray(a)
    if a.ndim == 1:
        return torch.tensor(a, dtype=dtype, device="cuda")
    return torch.tensor(np.ascontiguousarray(a.T), dtype=dtype, device="cuda")


def from_dev(t):
    a = t.detach().cpu().numpy().astype(np.float64)
    return a if a.ndim == 1 else np.asfortranarray(a.T)

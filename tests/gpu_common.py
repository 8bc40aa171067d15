"""Helpers shared by the GPU parity tests (test infrastructure)."""
import numpy as np
import pytest

_built = False


def lib():
    """Builds (once per session) and imports the package; skips without a GPU."""
    global _built
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if not _built:
        import __graft_entry__
        __graft_entry__.build()
        _built = True
    import paper_2203_04158_gb300 as G
    return G


def to_dev_u64(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).cuda()


def as_u64(t):
    return t.cpu().numpy().view(np.uint64)


def as_u32(t):
    return t.cpu().numpy().view(np.uint32)


def rel_inf(y, y_ref):
    y = np.asarray(y, dtype=np.float64)
    y_ref = np.asarray(y_ref, dtype=np.float64)
    return float(np.max(np.abs(y - y_ref)) / max(np.max(np.abs(y_ref)), 1e-300))

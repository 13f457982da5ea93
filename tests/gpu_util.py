"""Helpers shared by the GPU parity tests: building/loading the library, moving fields between
numpy and torch, and the relative L2 error used as the parity measure."""
import numpy as np
import pytest


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


# Tolerances (relative L2). complex64 fields: the relative field error bound 2e-5 of the target;
# complex128 fields: double-precision transforms, bounded well below 1e-10.
TOL_C64 = 2e-5
TOL_C128 = 1e-10
TOL_LOSS = 1e-4


def lib():
    """Builds (incrementally) and loads the CUDA library; skips when no GPU is present."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_08408_gb300 import build, xl
    build.build()
    xl.load()
    return xl


def to_dev(a, dtype):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


def to_np(t):
    return t.detach().cpu().numpy()

"""Shared helpers of the GPU parity tests (tensor transfer, error norms)."""
import numpy as np


def cuda():
    import torch
    if not torch.cuda.is_available():
        import pytest
        pytest.skip("no CUDA device")
    import paper_2105_11815_gb300 as pkg
    from paper_2105_11815_gb300 import build
    build.build()
    pkg.lib()
    return torch, pkg


def to_dev(torch, a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def rel_fro(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))

"""Helpers shared by the GPU tests: the library, tensors, errors."""
from __future__ import annotations

import numpy as np
import pytest


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1307_4370_gb300 import build

    build.build_library()
    return torch


def dev(a, torch):
    """numpy complex/float array -> CUDA tensor of the GPU storage type."""
    if np.iscomplexobj(a):
        return torch.tensor(np.ascontiguousarray(a).astype(np.complex64), device="cuda")
    return torch.tensor(np.ascontiguousarray(a).astype(np.float32), device="cuda")


def host(t):
    return t.detach().cpu().numpy().astype(np.complex128 if t.is_complex() else np.float64)


def rel_err(got, want) -> float:
    got = np.asarray(got, dtype=np.complex128)
    want = np.asarray(want, dtype=np.complex128)
    den = np.linalg.norm(want)
    return float(np.linalg.norm(got - want) / (den if den > 0 else 1.0))

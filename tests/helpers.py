"""Shared helpers for the GPU parity tests (no arithmetic of the method here)."""
import numpy as np
import pytest
import torch

# Error bounds: relative max-abs error max|c - c_ref| / max|c_ref| against the
# FP64 oracle, per arithmetic path.
TOL = {"fp64": 1e-12, "fp32": 1e-5, "bf16x3": 2e-6, "fixed": 1e-12}

requires_gpu = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")


def rel_err(got, ref) -> float:
    got = np.asarray(got)
    ref = np.asarray(ref)
    return float(np.max(np.abs(got.astype(np.complex128) - ref)) / max(np.max(np.abs(ref)), 1e-300))


def dev(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t: torch.Tensor) -> np.ndarray:
    torch.cuda.synchronize()
    return t.cpu().numpy()

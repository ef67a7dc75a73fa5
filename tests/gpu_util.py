"""Helpers shared by the GPU tests (no arithmetic of the method here)."""
import numpy as np
import pytest


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    return torch


def rel_err(got, ref):
    """max |got - ref| / max |ref| over the whole field (per array)."""
    return float(np.abs(np.asarray(got, np.float64) - ref).max() / max(np.abs(ref).max(), 1e-300))


def sine_basis(n):
    """Orthonormal eigenvectors of the 1D Dirichlet second difference:
    P[j][k] = sqrt(2/(n+1)) sin(pi (j+1)(k+1)/(n+1))."""
    j = np.arange(1, n + 1)
    return np.sqrt(2.0 / (n + 1)) * np.sin(np.pi * np.outer(j, j) / (n + 1))

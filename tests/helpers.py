"""Shared test helpers: host <-> device column-major storage and comparison metrics."""
import numpy as np


def dev(x):
    """numpy (rows x cols) -> cuda tensor holding its column-major storage (cols x rows)."""
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x).T)).to("cuda:0")


def host(t):
    """cuda storage tensor (cols x rows) -> numpy (rows x cols)."""
    return t.cpu().numpy().T


def subspace_sin(X, Y):
    """Largest principal-angle sine between span(X) and span(Y) (orthonormal columns)."""
    s = np.linalg.svd(np.conj(X.T) @ Y, compute_uv=False)
    return float(np.sqrt(max(0.0, 1.0 - np.min(s) ** 2)))

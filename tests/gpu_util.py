"""Shared helpers for the GPU parity tests (no method arithmetic)."""
import numpy as np
import pytest


def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def to_np(t):
    return t.detach().double().cpu().numpy()


def subspace_dist(X, Y):
    """||X X^T - Y Y^T||_2 for matrices with orthonormal columns."""
    Qx, _ = np.linalg.qr(X)
    Qy, _ = np.linalg.qr(Y)
    return np.linalg.norm(Qx @ Qx.T - Qy @ Qy.T, 2) if Qx.shape[0] <= 3000 else \
        np.sqrt(max(0.0, 1.0 - np.linalg.svd(Qx.T @ Qy, compute_uv=False).min() ** 2))

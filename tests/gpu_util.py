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


def subspace_tol(s_ref, k, rel_pert=3e-5):
    """(kk, tol): the leading kk singular vectors to compare and the bound on their
    subspace distance.  Wedin's theorem: a perturbation of relative size rel_pert
    (FP32 or split-BF16 arithmetic) moves the leading-kk singular subspace by at most
    about rel_pert * s_1 / (s_kk - s_{kk+1}); the bound never goes below 1e-3.
    kk < k so that s_{kk+1} is known; values below 1e-3 s_1 are left out."""
    import numpy as np
    s_ref = np.asarray(s_ref)
    kk = min(k - 1, int(np.sum(s_ref > 1e-3 * s_ref[0])))
    if kk < 1:
        return 0, 0.0
    gap = max(s_ref[kk - 1] - s_ref[kk], 1e-300)
    return kk, max(1e-3, rel_pert * s_ref[0] / gap)


def exact_resid_device(A, U, S, V, raw):
    """||A_c - U diag(S) V^T||_2 of a device matrix, from the FP64 Gram of the residual
    (torch eigvalsh on the device; measurement only).  Squaring costs u_64 (s_1/s)^2 of
    relative accuracy, far below the 1e-3 bars it is used with."""
    import torch
    m, n = A.shape
    Ud, Sd, Vd = U.double(), S.double(), V.double()
    mean = None if raw else A.double().mean(0)
    G = torch.zeros(n, n, dtype=torch.float64, device=A.device)
    for i in range(0, m, 8192):
        blk = A[i:i + 8192].double()
        if mean is not None:
            blk = blk - mean
        blk = blk - (Ud[i:i + 8192] * Sd) @ Vd.T
        G.addmm_(blk.T, blk)
    return float(torch.linalg.eigvalsh(G)[-1].clamp_min(0).sqrt().item())


def exact_singular_values_device(A, raw):
    """All singular values of A_c (descending) from the FP64 Gram on the device (measurement only)."""
    import torch
    m, n = A.shape
    mean = None if raw else A.double().mean(0)
    G = torch.zeros(n, n, dtype=torch.float64, device=A.device)
    for i in range(0, m, 8192):
        blk = A[i:i + 8192].double()
        if mean is not None:
            blk = blk - mean
        G.addmm_(blk.T, blk)
    return torch.linalg.eigvalsh(G).flip(0).clamp_min(0).sqrt().cpu().numpy()

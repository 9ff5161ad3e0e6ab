"""Seeded synthetic inputs for the randomized PCA of Szlam, Kluger & Tygert (2014).

This module only *constructs* test matrices.  It holds none of the PCA method's
arithmetic: no sketch, no renormalisation, no projection, no SVD of the
approximation.  Both the FP64 oracle (``oracle/``) and the CUDA path (through
the tests and ``bench.py``) draw their inputs from here, so that both sides see
the very same FP32 matrix.

Constructions follow the paper's own test matrices:

* dense ``A = U diag(sigma) V^T`` with Haar-distributed ``U`` and ``V`` obtained
  by orthonormalising i.i.d. N(0,1) vectors (Section 7, "Performance for dense
  matrices"); the QR used there is part of building the input, not of the
  method under test;
* the six spectra of Section 7 and the spectra of the benchmark workloads;
* the "importance of power iterations" matrix of Section 7 (Gaussian entries of
  mean sqrt(30/n), sign flipped where i*j is odd, 1-based);
* the diagonal matrices of Section 6 on which Lanczos (PROPACK) fails;
* power-law sparse matrices in CSR form standing in for the sparse collection of
  Section 8 (not available here);
* batches of Gaussian-kernel matrices exp(-|x_i - y_j|^2 / h) plus noise.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "spectrum_exp20", "spectrum_pow15", "spectrum_exp50", "spectrum_section7",
    "haar_dense_np", "haar_dense_torch", "e2_matrix_np", "e2_matrix_torch", "sym_dense_np", "sym_lowrank_np",
    "propack_diag",
    "powerlaw_csr", "kernel_matrix_np", "kernel_matrix_torch", "kernel_batch_specs", "KernelSpec",
    "WORKLOADS",
]


# ---------------------------------------------------------------------------
# spectra
# ---------------------------------------------------------------------------

def spectrum_exp20(r: int) -> np.ndarray:
    """sigma_j = exp(-j/20) for j <= 20, 1e-4 for j > 20 (1-based j)."""
    j = np.arange(1, r + 1, dtype=np.float64)
    return np.where(j <= 20, np.exp(-j / 20.0), 1e-4)


def spectrum_pow15(r: int, seed: int) -> np.ndarray:
    """sigma_j = j^-1.5 for j <= 200; tail i.i.d. uniform in [1e-5, 1e-4], sorted descending."""
    j = np.arange(1, r + 1, dtype=np.float64)
    s = j ** -1.5
    rng = np.random.default_rng(seed)
    tail = np.sort(rng.uniform(1e-5, 1e-4, size=max(r - 200, 0)))[::-1]
    s[200:] = tail
    return s


def spectrum_exp50(r: int) -> np.ndarray:
    """sigma_j = max(exp(-j/50), 1e-3) (1-based j)."""
    j = np.arange(1, r + 1, dtype=np.float64)
    return np.maximum(np.exp(-j / 50.0), 1e-3)


def spectrum_section7(kind: int, k: int, r: int, seed: int = 0) -> np.ndarray:
    """The six singular-value distributions of Section 7 (dense experiments).

    kind 1: 1/j.  kind 2: 1, then 2e-5 up to k, then 1e-5 (k+1)/j.
    kind 3: 10^(-5(j-1)/(k-1)) up to k, then 1e-5 (k+1)/j.
    kind 4: 10^(-5(j-1)/(k-1)) up to k, 1e-5 at k+1, zeros after.
    kind 5: 1e-5 + (1-1e-5)(k-j)/(k-1) up to k, then 1e-5 sqrt((k+1)/j).
    kind 6: |N(0,1)| draws (seeded), unsorted as drawn (the matrix
            construction does not need them sorted).
    For kinds 2-5 the spectral norm is 1 and the best rank-k error is 1e-5
    (kind 5 as printed has sigma_1 = 1 and sigma_{k+1} = 1e-5).
    """
    j = np.arange(1, r + 1, dtype=np.float64)
    if kind == 1:
        return 1.0 / j
    if kind == 2:
        s = np.where(j <= k, 2e-5, 1e-5 * (k + 1) / j)
        s[0] = 1.0
        return s
    if kind == 3:
        return np.where(j <= k, 10.0 ** (-5.0 * (j - 1) / (k - 1)), 1e-5 * (k + 1) / j)
    if kind == 4:
        s = np.where(j <= k, 10.0 ** (-5.0 * (j - 1) / (k - 1)), 0.0)
        if r > k:
            s[k] = 1e-5
        return s
    if kind == 5:
        return np.where(j <= k, 1e-5 + (1 - 1e-5) * (k - j) / (k - 1), 1e-5 * np.sqrt((k + 1) / j))
    if kind == 6:
        return np.abs(np.random.default_rng(seed).standard_normal(r))
    raise ValueError(kind)


# ---------------------------------------------------------------------------
# dense matrices with prescribed spectrum
# ---------------------------------------------------------------------------

def _haar_np(rng: np.random.Generator, rows: int, cols: int) -> np.ndarray:
    g = rng.standard_normal((rows, cols))
    q, r = np.linalg.qr(g)
    return q * np.sign(np.diag(r))[None, :]


def haar_dense_np(m: int, n: int, sigma: np.ndarray, seed: int, dtype=np.float32) -> np.ndarray:
    """A = U diag(sigma) V^T with Haar U (m x r), V (n x r), r = min(m, n); FP32 unless asked."""
    r = min(m, n)
    rng = np.random.default_rng(seed)
    u = _haar_np(rng, m, r)
    v = _haar_np(rng, n, r)
    return ((u * np.asarray(sigma[:r])[None, :]) @ v.T).astype(dtype)


def haar_dense_torch(m: int, n: int, sigma: np.ndarray, seed: int, device="cuda", return_colsum: bool = False):
    """Same construction on a torch device (for matrices too large for the host).

    The QR runs in FP32 on the device; the singular values of the stored FP32
    matrix therefore differ from ``sigma`` at the 1e-6 relative level, which is
    why exact reference singular values are recomputed from the stored matrix
    where that is affordable.  return_colsum: also return U^T 1 (FP64 host
    vector of length min(m, n), U the FP32 orthonormal factor used), the input
    metadata from which the spectrum of the column-centred matrix follows.
    """
    import torch
    r = min(m, n)
    g = torch.Generator(device=device)
    g.manual_seed(seed)

    def haar(rows, cols):
        x = torch.randn(rows, cols, generator=g, device=device, dtype=torch.float32)
        q, rr = torch.linalg.qr(x)
        q.mul_(torch.sign(torch.diagonal(rr))[None, :])
        del x, rr
        return q

    u = haar(m, r)
    colsum = None
    if return_colsum:
        cs = torch.zeros(r, dtype=torch.float64, device=device)
        for i in range(0, m, 8192):
            cs += u[i:i + 8192].double().sum(0)
        colsum = cs.cpu().numpy()
    u.mul_(torch.as_tensor(np.asarray(sigma[:r]), dtype=torch.float32, device=device)[None, :])
    v = haar(n, r)
    a = u @ v.T
    del u, v
    return (a.contiguous(), colsum) if return_colsum else a.contiguous()


def e2_matrix_np(n: int, seed: int) -> np.ndarray:
    """n x n i.i.d. N(sqrt(30/n), 1), sign flipped where i*j is odd (1-based), FP32."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((n, n)) + math.sqrt(30.0 / n)
    i = np.arange(1, n + 1)
    odd = ((i[:, None] * i[None, :]) % 2) == 1
    a[odd] = -a[odd]
    return a.astype(np.float32)


def e2_matrix_torch(n: int, seed: int, device="cuda", rows_per_chunk: int = 4096):
    """The same law on a torch device (torch's generator, row chunks), FP32: N(sqrt(30/n), 1)
    entries, sign flipped where i*j is odd (1-based i, j: both odd)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    a = torch.empty(n, n, dtype=torch.float32, device=device)
    mu = math.sqrt(30.0 / n)
    for r0 in range(0, n, rows_per_chunk):
        r1 = min(n, r0 + rows_per_chunk)
        blk = torch.randn(r1 - r0, n, generator=g, device=device, dtype=torch.float32)
        blk += mu
        # 1-based row r0 + t + 1 is odd when the 0-based row r0 + t is even
        blk[r0 % 2::2, 0::2] *= -1.0
        a[r0:r1] = blk
        del blk
    return a


def sym_dense_np(n: int, lam, seed: int, dtype=np.float32) -> np.ndarray:
    """Self-adjoint A = Q diag(lam) Q^T with Haar Q (n x n), symmetrised exactly after
    rounding ((A + A^T) / 2 in the target precision is symmetric bit for bit)."""
    rng = np.random.default_rng(seed)
    q = _haar_np(rng, n, n)
    a = ((q * np.asarray(lam, dtype=np.float64)[None, :]) @ q.T).astype(dtype)
    return ((a + a.T) / dtype(2)).astype(dtype)


def sym_lowrank_np(n: int, lam_top, tail: float, seed: int, psd: bool = False, dtype=np.float32) -> np.ndarray:
    """Large self-adjoint A without an n x n QR: Q diag(lam_top) Q^T (Q Haar, n x r) plus a
    tail -- tail * I when psd (nonnegative definite, flat tail), else a symmetric
    Gaussian matrix scaled to spectral norm about tail (semicircle radius 2 s sqrt(n))."""
    rng = np.random.default_rng(seed)
    lam_top = np.asarray(lam_top, dtype=np.float64)
    q = _haar_np(rng, n, lam_top.size)
    a = (q * lam_top[None, :]) @ q.T
    if psd:
        a[np.arange(n), np.arange(n)] += tail
    else:
        g = rng.standard_normal((n, n)) * (tail / (2.0 * math.sqrt(2.0 * n)))
        a += g + g.T
    a = a.astype(dtype)
    return ((a + a.T) / dtype(2)).astype(dtype)


def propack_diag(size: int) -> np.ndarray:
    """Section 6: diag(1, 1, 1, .999 (17 times), 0, ...) of the given size, FP32."""
    d = np.zeros(size)
    d[:3] = 1.0
    d[3:20] = 0.999
    return np.diag(d).astype(np.float32)


# ---------------------------------------------------------------------------
# sparse power-law matrices (CSR)
# ---------------------------------------------------------------------------

def powerlaw_csr(m: int, n: int, nnz: int, exponent: float = 2.1, rank: int = 30,
                 seed: int = 0, boost=(10.0, 100.0)):
    """CSR matrix with power-law row and column degrees plus a planted rank-``rank`` part.

    Chung-Lu style: rows are drawn with probability proportional to
    w_i = (i + 1)^(-1/(exponent-1)), columns likewise; duplicate (row, col)
    pairs are dropped and further draws top the set up to exactly ``nnz``
    distinct entries.  Values are N(0,1) plus sum_r s_r x_ir y_jr on the
    pattern only, with x, y Gaussian (columns scaled to unit norm) and s_r
    log-spaced between boost[0] and boost[1] times the bulk scale
    sqrt(max row degree) + sqrt(max column degree).

    Returns (row_ptr int32[m+1], col_idx int32[nnz], val float32[nnz]) with
    column indices sorted within each row.
    """
    rng = np.random.default_rng(seed)
    alpha = 1.0 / (exponent - 1.0)
    pr = (np.arange(1, m + 1, dtype=np.float64)) ** (-alpha)
    pc = (np.arange(1, n + 1, dtype=np.float64)) ** (-alpha)
    pr /= pr.sum()
    pc /= pc.sum()
    # random relabelling so that heavy rows/columns are spread over the index range
    rperm = rng.permutation(m)
    cperm = rng.permutation(n)
    keys = np.empty(0, dtype=np.int64)
    while keys.size < nnz:
        need = int((nnz - keys.size) * 1.3) + 1024
        r = rperm[rng.choice(m, size=need, p=pr)]
        c = cperm[rng.choice(n, size=need, p=pc)]
        keys = np.unique(np.concatenate([keys, r.astype(np.int64) * n + c]))
    if keys.size > nnz:
        keys = np.sort(rng.choice(keys, size=nnz, replace=False))
    rows = (keys // n).astype(np.int64)
    cols = (keys % n).astype(np.int64)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    deg_r = np.diff(row_ptr)
    deg_c = np.bincount(cols, minlength=n)
    bulk = math.sqrt(deg_r.max()) + math.sqrt(deg_c.max())
    x = rng.standard_normal((m, rank))
    y = rng.standard_normal((n, rank))
    x /= np.linalg.norm(x, axis=0, keepdims=True)
    y /= np.linalg.norm(y, axis=0, keepdims=True)
    s = bulk * np.geomspace(boost[1], boost[0], rank)
    # planted part on the pattern: sum_r s_r x[row, r] y[col, r], in chunks
    val = rng.standard_normal(nnz)
    chunk = 1 << 20
    for a in range(0, nnz, chunk):
        b = min(a + chunk, nnz)
        val[a:b] += np.einsum("ir,ir,r->i", x[rows[a:b]], y[cols[a:b]], s)
    return row_ptr.astype(np.int32), cols.astype(np.int32), val.astype(np.float32)


# ---------------------------------------------------------------------------
# batches of Gaussian-kernel matrices
# ---------------------------------------------------------------------------

@dataclass
class KernelSpec:
    m: int
    n: int
    h: float
    seed: int


def kernel_batch_specs(count: int, seed: int, m_range=(256, 8192), n_range=(64, 1024)):
    """Shapes and bandwidths of a batch: m, n log-uniform (rounded), h log-uniform in [0.05, 1]."""
    rng = np.random.default_rng(seed)
    lm = rng.uniform(math.log(m_range[0]), math.log(m_range[1]), size=count)
    ln = rng.uniform(math.log(n_range[0]), math.log(n_range[1]), size=count)
    lh = rng.uniform(math.log(0.05), math.log(1.0), size=count)
    seeds = rng.integers(0, 2**31 - 1, size=count)
    return [KernelSpec(int(round(math.exp(a))), int(round(math.exp(b))), float(math.exp(c)), int(d))
            for a, b, c, d in zip(lm, ln, lh, seeds)]


def kernel_matrix_torch(spec: KernelSpec, device="cuda", noise_var: float = 1e-4):
    """Same family on a torch device (torch's generator, seeded by spec.seed), FP32."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(spec.seed)
    x = torch.rand(spec.m, 3, generator=g, device=device, dtype=torch.float32)
    y = torch.rand(spec.n, 3, generator=g, device=device, dtype=torch.float32)
    d2 = (x * x).sum(1)[:, None] + (y * y).sum(1)[None, :] - 2.0 * (x @ y.T)
    a = torch.exp(-d2.clamp_min(0.0) / spec.h)
    a += math.sqrt(noise_var) * torch.randn(spec.m, spec.n, generator=g, device=device, dtype=torch.float32)
    return a


def kernel_matrix_np(spec: KernelSpec, noise_var: float = 1e-4) -> np.ndarray:
    """A_ij = exp(-|x_i - y_j|^2 / h) + N(0, noise_var), x, y ~ U[0,1]^3, FP32."""
    rng = np.random.default_rng(spec.seed)
    x = rng.uniform(size=(spec.m, 3))
    y = rng.uniform(size=(spec.n, 3))
    d2 = ((x[:, None, :] - y[None, :, :]) ** 2).sum(-1)
    a = np.exp(-d2 / spec.h) + math.sqrt(noise_var) * rng.standard_normal((spec.m, spec.n))
    return a.astype(np.float32)


# ---------------------------------------------------------------------------
# the benchmark workloads (shapes and parameters), named by what they are
# ---------------------------------------------------------------------------

WORKLOADS = {
    # name: (m, n, k, l, its, raw, spectrum builder, seed)
    "dense_2000x1000_k10": dict(m=2000, n=1000, k=10, l=12, its=2, raw=False,
                                spectrum=lambda r: spectrum_exp20(r), seed=1235),
    # its_at_bar: the smallest its whose PCA of this (seeded, fixed) matrix meets resid <=
    # 1.1 sigma_{k+1}, as bench.py's accuracy search finds it on the GPU (resid / sigma_101 =
    # 1.179, 1.124, 1.088 at its = 2, 3, 4); the host reference times the oracle at it too
    "dense_100000x2000_k100": dict(m=100000, n=2000, k=100, l=102, its=2, raw=False, its_at_bar=4,
                                   spectrum=lambda r: spectrum_pow15(r, 1236), seed=1236),
    "dense_200000x20000_k200": dict(m=200000, n=20000, k=200, l=210, its=2, raw=False,
                                    spectrum=lambda r: spectrum_exp50(r), seed=1237),
    # a quarter-size version of the 100000 x 2000 workload (A = 200 MB, still larger
    # than L2) for profiler captures that must stay small
    "dense_25000x2000_k100": dict(m=25000, n=2000, k=100, l=102, its=2, raw=False,
                                  spectrum=lambda r: spectrum_pow15(r, 1236), seed=1238),
    # Section 7's importance-of-power-iterations matrix: n x n i.i.d. N(sqrt(30/n), 1), signs
    # flipped where i*j is odd; rank 4, l = k + 2, its swept over 0, 2, 4; A itself (raw)
    # its_at_bar = 3: resid / sigma_5 = 1.79 at its = 2, 1.07 at its = 3
    "e2_gaussian_100000_k4": dict(kind="e2", m=100000, n=100000, k=4, l=6, its=2, raw=True, its_sweep=(0, 2, 4),
                                  its_at_bar=3, seed=1243),
    "e2_gaussian_20000_k4": dict(kind="e2", m=20000, n=20000, k=4, l=6, its=2, raw=True, its_sweep=(0, 2, 4),
                                 seed=1244),
    # sparse: power-law row/column degrees (exponent 2.1), N(0,1) values plus a planted
    # rank-30 part on the pattern
    "csr_1000000x100000_k30": dict(kind="csr", m=1000000, n=100000, nnz=10000000, exponent=2.1, rank=30,
                                   k=30, l=32, its=4, raw=True, seed=1239),
    "csr_100000x10000_k30": dict(kind="csr", m=100000, n=10000, nnz=1000000, exponent=2.1, rank=30,
                                 k=30, l=32, its=4, raw=True, seed=1240),
    # batched: Gaussian-kernel matrices exp(-|x_i - y_j|^2 / h) + N(0, 1e-4), m and n
    # log-uniform, x, y ~ U[0,1]^3, h log-uniform in [0.05, 1]
    "batched_4096_kernel_k16": dict(kind="batched", count=4096, m_range=(256, 8192), n_range=(64, 1024),
                                    k=16, l=20, its=2, raw=False, seed=1241),
    "batched_512_kernel_k16": dict(kind="batched", count=512, m_range=(256, 8192), n_range=(64, 1024),
                                   k=16, l=20, its=2, raw=False, seed=1242),
}

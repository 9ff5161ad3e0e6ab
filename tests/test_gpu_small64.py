"""The FP64 l x l path (RPCA_PREC_SMALL_FP64): the Cholesky factors and inverses of the
CholeskyQR renormalisations, the accumulated factor R of B^* = Q2 R and the SVD of
R^T (FP32 Jacobi refined to FP64 accuracy) in FP64.

* The small SVD alone (rpca_small_svd) reaches FP64 accuracy on l x l matrices with
  graded, distinct singular values: an FP32 SVD could not pass these bars.
* Whole PCAs with the option match the FP64 oracle to the same bars as the FP32
  l x l path, in both pass precisions, on dense, CSR, self-adjoint and Nystrom input.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
import synth as S
from gpu_util import cuda, subspace_dist, subspace_tol, to_dev, to_np

pytestmark = pytest.mark.gpu


def _graded(l, seed, lo=1e-6):
    rng = np.random.default_rng(seed)
    u, _ = np.linalg.qr(rng.standard_normal((l, l)))
    v, _ = np.linalg.qr(rng.standard_normal((l, l)))
    s = np.geomspace(1.0, lo, l)
    return (u * s) @ v.T, s


@pytest.mark.parametrize("l", [1, 12, 50, 102, 128, 150, 224])
def test_small_svd_reaches_fp64_accuracy(l):
    cuda()
    import torch
    import paper_1412_3510_gb300 as rp
    M, s = _graded(l, l)
    Sg, W, Z = (x.cpu().numpy() for x in rp.rpca_small_svd(torch.from_numpy(M).cuda()))
    I = np.eye(l)
    assert np.all(np.abs(Sg - s) <= 1e-13 * s[0] + 1e-9 * s), np.max(np.abs(Sg - s) / s)
    assert np.linalg.norm(W.T @ W - I, 2) < 1e-13 * l
    assert np.linalg.norm(Z.T @ Z - I, 2) < 1e-13 * l
    assert np.linalg.norm(M - (W * Sg) @ Z.T, 2) < 1e-13 * l * s[0]
    # the oracle's one-sided Jacobi on the same matrix
    _, so, _ = O.jacobi_svd(M)
    assert np.all(np.abs(Sg - so) <= 1e-13 * so[0] + 1e-9 * so)


def _check(Ug, sg, Uo, so, k):
    assert np.all(np.diff(sg) <= 0)
    assert np.all(np.abs(sg - so) <= 1e-4 * so + 2e-6 * so[0]), (np.abs(sg - so) / so).max()
    assert np.linalg.norm(Ug.T @ Ug - np.eye(k), 2) < 1e-4
    kk, tol = subspace_tol(so, k)
    if kk:
        assert subspace_dist(Ug[:, :kk], Uo[:, :kk]) < max(1e-3, tol)


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
@pytest.mark.parametrize("m,n,k,l,its,raw", [
    (600, 400, 10, 12, 2, False),
    (1000, 500, 100, 150, 1, False),      # l > 128: the shared-memory Jacobi
    (20000, 300, 40, 50, 2, False),       # tall: tensor-core Gram and products
    (333, 257, 5, 7, 0, True),
])
def test_dense_small_fp64_parity(m, n, k, l, its, raw, precision):
    cuda()
    import paper_1412_3510_gb300 as rp
    sig = np.exp(-np.arange(1, min(m, n) + 1) / max(4.0, l / 2.0))
    A = S.haar_dense_np(m, n, sig, seed=m + n)
    if not raw:
        A = A + np.float32(0.3)
    U, Sg, V = rp.rpca_dense(to_dev(A), k, l, its=its, raw=raw, seed=4, precision=precision, small_fp64=True)
    Uo, so, Vo = O.rpca(A, k, l, its, raw=raw, seed=4)
    _check(to_np(U), to_np(Sg), Uo, so, k)
    _check(to_np(V), to_np(Sg), Vo, so, k)
    # the same PCA with the FP32 l x l path agrees to the noise of the passes: FP32 FFMA, or
    # 16 significant bits per factor in the split-BF16 form (the two runs' blocks differ in
    # their last bits, and so do their BF16 splits)
    _, S32, _ = rp.rpca_dense(to_dev(A), k, l, its=its, raw=raw, seed=4, precision=precision)
    rtol = 2e-5 if precision == "fp32" else 6e-5
    assert np.all(np.abs(to_np(Sg) - to_np(S32)) <= rtol * to_np(S32) + 2e-6 * so[0])


def test_csr_sym_nystrom_small_fp64_parity():
    cuda()
    import torch
    import paper_1412_3510_gb300 as rp
    rp_, ci, va = S.powerlaw_csr(3000, 1500, 40000, exponent=2.1, rank=8, seed=5)
    csr = sp.csr_matrix((va, ci, rp_), shape=(3000, 1500))
    dev = [torch.from_numpy(x).cuda() for x in (rp_, ci, va)]
    U, Sg, V = rp.rpca_csr(*dev, csr.shape, 8, 10, its=3, raw=True, seed=11, small_fp64=True)
    Uo, so, Vo = O.rpca(csr, 8, 10, 3, raw=True, seed=11)
    _check(to_np(U), to_np(Sg), Uo, so, 8)
    j = np.arange(1, 401)
    A = S.sym_dense_np(400, np.exp(-j / 6.0) * np.where(j % 3 == 0, -1.0, 1.0), 9)
    U, Sg, V = rp.rpca_sym(to_dev(A), 8, 10, its=3, seed=2, small_fp64=True)
    Uo, so, Vo = O.rpca_sym(A, 8, 10, 3, seed=2)
    _check(to_np(U), to_np(Sg), Uo, so, 8)
    P = S.sym_dense_np(400, 1.0 / j ** 2, 3)
    U, Sg = rp.rpca_nystrom(to_dev(P), 8, 10, its=2, seed=2, small_fp64=True)
    Uo, so = O.nystrom(P, 8, 10, 2, seed=2)
    _check(to_np(U), to_np(Sg), Uo, so, 8)

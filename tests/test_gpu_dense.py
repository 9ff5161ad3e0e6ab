"""Parity of the CUDA dense path (rpca_dense through the C ABI) with the FP64 oracle.

Both sides get the same FP32 matrix and the same Philox seed; the oracle draws
Omega in FP64, the GPU in FP32 (identical uniforms, FP32 log/sincos).  The
bar (FP32 path): singular values within 1e-4 relative (plus an absolute floor
of 1e-6 ||A|| for values at FP32 rounding level), singular subspaces within
1e-3 or the Wedin bound for their spectral gap (gpu_util.subspace_tol), and
U, V orthonormal to 1e-4.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
import synth as S
from gpu_util import cuda, subspace_dist, subspace_tol, to_dev, to_np

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _check_parity(A, k, l, its, raw, seed, sig_rtol=1e-4, sub_tol=1e-3, **kw):
    cuda()
    import paper_1412_3510_gb300 as rp
    U, Sg, V = rp.rpca_dense(to_dev(A), k, l, its=its, raw=raw, seed=seed, **kw)
    Ug, sg, Vg = to_np(U), to_np(Sg), to_np(V)
    Uo, so, Vo = O.rpca(A, k, l, its, raw=raw, seed=seed)
    floor = 1e-6 * so[0]
    assert np.all(np.abs(sg - so) <= sig_rtol * so + floor), (np.abs(sg - so) / so).max()
    assert np.all(np.diff(sg) <= 0)
    assert np.linalg.norm(Ug.T @ Ug - np.eye(k), 2) < 1e-4
    assert np.linalg.norm(Vg.T @ Vg - np.eye(k), 2) < 1e-4
    # subspaces of the leading singular vectors whose values are above the noise floor
    kk, tol = subspace_tol(so, k)
    if kk:
        assert subspace_dist(Ug[:, :kk], Uo[:, :kk]) < max(sub_tol, tol)
        assert subspace_dist(Vg[:, :kk], Vo[:, :kk]) < max(sub_tol, tol)
    # sign convention: largest-|entry| of every V column is positive
    idx = np.argmax(np.abs(Vg), axis=0)
    assert np.all(Vg[idx, np.arange(k)] > 0)
    return Ug, sg, Vg, (Uo, so, Vo)


CASES = [
    # m, n, k, l, its, raw          (ragged sizes, wide and tall, its 0..3, l = min(m, n), l = 1)
    (333, 257, 5, 7, 2, False),
    (257, 333, 5, 7, 1, True),
    (600, 400, 10, 12, 2, False),
    (129, 129, 8, 10, 0, False),
    (1000, 300, 30, 40, 3, False),
    (50, 40, 10, 40, 1, True),
    (100, 80, 1, 1, 2, False),
    (2000, 1000, 10, 12, 2, False),
    (1000, 500, 200, 224, 1, False),
    (4097, 130, 20, 33, 2, False),
]


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
@pytest.mark.parametrize("m,n,k,l,its,raw", CASES)
def test_dense_parity(m, n, k, l, its, raw, precision):
    sig = np.exp(-np.arange(1, min(m, n) + 1) / max(4.0, l / 2.0))
    A = S.haar_dense_np(m, n, sig, seed=m * 7 + n)
    if not raw:
        A = A + np.float32(0.3) * np.random.default_rng(m).standard_normal(n).astype(np.float32)[None, :]
    _check_parity(A, k, l, its, raw, seed=m + n + k, precision=precision)


# tall blocks (>= 16384 rows): the renormalisations' Gram matrices and Y R^-1 products
# and the U lift run on the tensor cores in three-piece split BF16; lp <= 128 takes the
# tensor-core Gram, wider blocks the SIMT Gram with the tensor-core products
TALL_CASES = [
    (20000, 300, 40, 50, 2, False),
    (33333, 500, 100, 120, 1, False),     # lp = 128, the widest tensor-core Gram
    (16384, 200, 10, 12, 3, True),
    (40000, 257, 150, 160, 1, False),     # lp = 168: SIMT Gram, tensor-core products
    (17001, 300, 5, 8, 0, True),          # its = 0
]


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
@pytest.mark.parametrize("m,n,k,l,its,raw", TALL_CASES)
def test_dense_tall_parity(m, n, k, l, its, raw, precision):
    sig = np.exp(-np.arange(1, min(m, n) + 1) / max(4.0, l / 2.0))
    A = S.haar_dense_np(m, n, sig, seed=m * 7 + n)
    if not raw:
        A = A + np.float32(0.3) * np.random.default_rng(m).standard_normal(n).astype(np.float32)[None, :]
    _check_parity(A, k, l, its, raw, seed=m + n + k, precision=precision)


@pytest.mark.parametrize("raw", [True, False])
def test_exact_low_rank_recovery_tall(raw):
    """Rank r < l on 20000 rows: the final CholeskyQR shifts and runs its third round
    on the tensor cores (and skips it in the other case, an identity copy)."""
    cuda()
    import paper_1412_3510_gb300 as rp
    rng = np.random.default_rng(5)
    r = 9 if raw else 8
    A = (rng.standard_normal((20000, r)) @ rng.standard_normal((r, 300))).astype(np.float32)
    if not raw:
        A += np.float32(2.0)
    # Bars: the Gram of the 20000-row block runs on the tensor cores, whose FP32
    # accumulation drifts by up to ~2e-6 relative (256-row chains), so Q and U = Q W are
    # orthonormal to a few 1e-6 and the reconstruction error is of that order
    # (measured 1.2e-6 .. 2.5e-6 in both pass precisions; 4e-6 = 67 u_32).
    for l in (11, 9):
        U, Sg, V = rp.rpca_dense(to_dev(A), 9, l, its=1, raw=raw, seed=4)
        Ac = A.astype(np.float64) - (0 if raw else A.astype(np.float64).mean(0))
        E = Ac - (to_np(U) * to_np(Sg)) @ to_np(V).T
        assert np.linalg.norm(E, 2) / np.linalg.norm(Ac, 2) < 4e-6, l
        Ug, Vg = to_np(U), to_np(V)
        assert np.linalg.norm(Ug.T @ Ug - np.eye(9), 2) < 1e-5
        assert np.linalg.norm(Vg.T @ Vg - np.eye(9), 2) < 1e-5


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
@pytest.mark.parametrize("m,n,k,l,its,raw", [c for c in CASES if c[3] <= 160] + [(20000, 300, 40, 150, 2, False)])
def test_dense_lu_renorm_parity(m, n, k, l, its, raw, precision):
    """Section 5's LU renormalisation (tall-skinny LU, tournament pivoting) against the
    oracle's partial-pivoting LU: the span after every renormalisation is the same, so
    the outputs agree to the same bar."""
    sig = np.exp(-np.arange(1, min(m, n) + 1) / max(4.0, l / 2.0))
    A = S.haar_dense_np(m, n, sig, seed=m * 7 + n)
    if not raw:
        A = A + np.float32(0.3) * np.random.default_rng(m).standard_normal(n).astype(np.float32)[None, :]
    _check_parity(A, k, l, its, raw, seed=m + n + k, precision=precision, renorm="lu")


def test_dense_lu_rank_deficient_and_unsupported_width():
    cuda()
    import paper_1412_3510_gb300 as rp
    # rank 3 with l = 8: the LU meets zero pivots, which count as shifts; the leading
    # triplets still match the oracle
    rng = np.random.default_rng(2)
    A = (rng.standard_normal((700, 3)) @ rng.standard_normal((3, 90))).astype(np.float32)
    U, Sg, V = rp.rpca_dense(to_dev(A), 3, 8, its=2, raw=True, seed=5, renorm="lu")
    _, so, _ = O.rpca(A, 3, 8, 2, raw=True, seed=5)
    assert np.all(np.abs(to_np(Sg) - so) <= 1e-4 * so)
    # the tall-skinny LU holds 2l x (l + 1) entries per node: l > 160 is refused
    B = to_dev(rng.standard_normal((400, 200)).astype(np.float32))
    with pytest.raises(rp.RpcaError) as e:
        rp.rpca_dense(B, 150, 170, its=1, renorm="lu")
    assert e.value.code == -7


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_dense_first_workload_full_size(precision):
    w = S.WORKLOADS["dense_2000x1000_k10"]
    A = S.haar_dense_np(w["m"], w["n"], w["spectrum"](min(w["m"], w["n"])), w["seed"])
    _check_parity(A, w["k"], w["l"], w["its"], w["raw"], seed=1, precision=precision)


def test_section6_examples_on_gpu():
    with open(os.path.join(GOLDEN, "section6_lanczos_failures.json")) as f:
        gold = json.load(f)
    cuda()
    import paper_1412_3510_gb300 as rp
    for case in gold["cases"]:
        A = S.propack_diag(case["size"])
        k = case["k"]
        _, Sg, _ = rp.rpca_dense(to_dev(A), k, k + 2, its=2, raw=True, seed=17)
        assert np.allclose(to_np(Sg), np.array(case["expect_sorted"], dtype=np.float64), atol=2e-6, rtol=0)


@pytest.mark.parametrize("raw", [True, False])
def test_exact_low_rank_recovery(raw):
    cuda()
    import paper_1412_3510_gb300 as rp
    rng = np.random.default_rng(3)
    r = 9 if raw else 8
    A = (rng.standard_normal((700, r)) @ rng.standard_normal((r, 300))).astype(np.float32)
    if not raw:
        A += np.float32(2.0)
    U, Sg, V = rp.rpca_dense(to_dev(A), 9, 11, its=1, raw=raw, seed=4)
    Ac = A.astype(np.float64) - (0 if raw else A.astype(np.float64).mean(0))
    E = Ac - (to_np(U) * to_np(Sg)) @ to_np(V).T
    assert np.linalg.norm(E, 2) / np.linalg.norm(Ac, 2) < 2e-6


def test_deterministic_and_strided_inputs():
    cuda()
    import torch
    import paper_1412_3510_gb300 as rp
    A = S.haar_dense_np(500, 300, np.exp(-np.arange(1, 301) / 8.0), seed=2)
    big = torch.zeros(500, 307, dtype=torch.float32, device="cuda")
    big[:, :300] = to_dev(A)
    Av = big[:, :300]                      # lda = 307, unaligned rows
    a = rp.rpca_dense(Av, 6, 9, its=2, seed=5)
    b = rp.rpca_dense(Av, 6, 9, its=2, seed=5)
    c = rp.rpca_dense(to_dev(A), 6, 9, its=2, seed=5)
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    for x, y in zip(a, c):
        assert torch.allclose(x, y, rtol=1e-5, atol=1e-6)
    # strided outputs (ldu, ldv > k)
    U = torch.full((500, 10), 7.0, device="cuda")
    V = torch.full((300, 10), 7.0, device="cuda")
    Sx = torch.empty(6, device="cuda")
    rp.rpca_dense(to_dev(A), 6, 9, its=2, seed=5, out=(U[:, :6], Sx, V[:, :6]))
    assert torch.allclose(U[:, :6], c[0], atol=1e-6) and torch.all(U[:, 6:] == 7.0)
    assert torch.allclose(V[:, :6], c[2], atol=1e-6) and torch.all(V[:, 6:] == 7.0)


def test_caller_omega_and_weights():
    cuda()
    import torch
    import paper_1412_3510_gb300 as rp
    A = S.haar_dense_np(400, 200, np.exp(-np.arange(1, 201) / 6.0), seed=9)
    Om = O.gaussian_omega(200, 8, seed=3).astype(np.float32)
    d = np.linspace(0.5, 2.0, 200).astype(np.float32)
    U, Sg, V = rp.rpca_dense(to_dev(A), 6, 8, its=1, omega=to_dev(Om), col_weights=to_dev(d))
    _, so, _ = O.rpca(A, 6, 8, 1, omega=Om.astype(np.float64) * d[:, None].astype(np.float64))
    assert np.allclose(to_np(Sg), so, rtol=1e-4, atol=1e-6 * so[0])


def test_invalid_arguments_raise():
    cuda()
    import paper_1412_3510_gb300 as rp
    A = to_dev(np.ones((20, 10), dtype=np.float32))
    with pytest.raises(rp.RpcaError):
        rp.rpca_dense(A, 5, 11)        # l > min(m, n)
    with pytest.raises(rp.RpcaError):
        rp.rpca_dense(A, 5, 4)         # l < k
    with pytest.raises(rp.RpcaError):
        rp.rpca_dense(A, 5, 6, its=-1)


def test_nonfinite_input_reports_status():
    cuda()
    import paper_1412_3510_gb300 as rp
    A = np.random.default_rng(0).standard_normal((64, 32)).astype(np.float32)
    A[5, 7] = np.nan
    with pytest.raises(rp.RpcaError) as e:
        rp.rpca_dense(to_dev(A), 4, 6)
    assert e.value.code == -4

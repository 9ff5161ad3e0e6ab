"""Pins for the oracle's building blocks (Section 5 renormalisations and centring; Eq. i3 SVD).

Each is checked against an independent library routine (scipy's LU, numpy's
QR and SVD) or against a definition the routine must satisfy exactly.
"""
import numpy as np
import pytest
import scipy.linalg

import oracle as O


def _rand(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


@pytest.mark.parametrize("m,l", [(50, 7), (333, 12), (40, 40), (1000, 33)])
def test_lu_matches_scipy_partial_pivoting(m, l):
    Y = _rand((m, l), m + l)
    Q, R = O.lu_renorm(Y)
    P, L, U = scipy.linalg.lu(Y)          # Y = P L U, LAPACK getrf pivoting
    assert np.allclose(Q, P @ L, atol=1e-13, rtol=0)
    assert np.allclose(R, U, atol=1e-12, rtol=1e-13)
    assert np.allclose(Q @ R, Y, atol=1e-12)
    assert np.max(np.abs(Q)) <= 1.0 + 1e-15
    assert np.allclose(R, np.triu(R))


def test_lu_ties_take_first_row_and_zero_pivot():
    Y = np.array([[1.0, 2.0], [-1.0, 5.0], [1.0, 1.0]])
    Q, R = O.lu_renorm(Y)
    assert R[0, 0] == 1.0                 # first of the tied |1| entries
    Z = np.zeros((4, 2))
    Z[:, 1] = [1, 2, 3, 4]
    Q, R = O.lu_renorm(Z)                 # zero first column: no division
    assert np.all(np.isfinite(Q)) and np.allclose(Q @ R, Z)


@pytest.mark.parametrize("m,l", [(60, 5), (500, 40), (17, 17)])
def test_householder_qr(m, l):
    Y = _rand((m, l), 3 * m + l)
    Q, R = O.householder_qr(Y)
    assert np.allclose(Q.T @ Q, np.eye(l), atol=1e-13)
    assert np.allclose(Q @ R, Y, atol=1e-12)
    assert np.allclose(R, np.triu(R))
    Qn, Rn = np.linalg.qr(Y)
    assert np.allclose(np.abs(R), np.abs(Rn), atol=1e-12)
    assert np.allclose(np.abs(Q.T @ Qn), np.eye(l), atol=1e-12)


@pytest.mark.parametrize("shape", [(9, 9), (40, 13), (13, 40), (120, 120), (300, 31)])
def test_jacobi_svd_matches_numpy(shape):
    M = _rand(shape, sum(shape))
    U, s, V = O.jacobi_svd(M)
    sn = np.linalg.svd(M, compute_uv=False)
    assert np.allclose(s, sn, rtol=1e-13, atol=1e-14 * sn[0])
    r = min(shape)
    assert np.allclose(U.T @ U, np.eye(r), atol=1e-13)
    assert np.allclose(V.T @ V, np.eye(r), atol=1e-13)
    assert np.allclose((U * s) @ V.T, M, atol=1e-12 * sn[0])
    assert np.all(np.diff(s) <= 0)


def test_jacobi_svd_closed_forms():
    # diagonal: singular values are |d| sorted
    d = np.array([0.3, -2.0, 1.5, 0.0, 7.0])
    U, s, V = O.jacobi_svd(np.diag(d))
    assert np.allclose(s, [7.0, 2.0, 1.5, 0.3, 0.0], atol=1e-15)
    assert np.allclose(U.T @ U, np.eye(5), atol=1e-14)
    # 2x2 upper triangular [[a, b], [0, c]]: s1^2 + s2^2 = a^2+b^2+c^2, s1 s2 = |a c|
    a, b, c = 3.0, -4.0, 0.5
    _, s, _ = O.jacobi_svd(np.array([[a, b], [0.0, c]]))
    T, D = a * a + b * b + c * c, abs(a * c)
    s1 = np.sqrt((T + np.sqrt(T * T - 4 * D * D)) / 2)
    s2 = np.sqrt((T - np.sqrt(T * T - 4 * D * D)) / 2)
    assert np.allclose(s, [s1, s2], rtol=1e-14)


def test_jacobi_svd_rank_deficient():
    rng = np.random.default_rng(8)
    M = rng.standard_normal((30, 4)) @ rng.standard_normal((4, 12))
    U, s, V = O.jacobi_svd(M)
    assert np.all(s[4:] < 1e-13 * s[0])
    assert np.allclose(U.T @ U, np.eye(12), atol=1e-12)
    assert np.allclose((U * s) @ V.T, M, atol=1e-12 * s[0])


@pytest.mark.parametrize("q", [1, 2, 5, 8, 13])
def test_round_robin_covers_every_pair_once(q):
    steps = O.round_robin_steps(q)
    seen = []
    for P, Qc in steps:
        cols = np.concatenate([P, Qc])
        assert len(set(cols.tolist())) == cols.size      # disjoint within a step
        assert np.all(P < Qc)
        seen += list(zip(P.tolist(), Qc.tolist()))
    assert sorted(seen) == [(i, j) for i in range(q) for j in range(i + 1, q)]


def test_implicit_centring_equals_explicit():
    rng = np.random.default_rng(4)
    A = rng.standard_normal((70, 30)) + 5.0 * rng.standard_normal(30)[None, :]
    X = rng.standard_normal((30, 6))
    Y = rng.standard_normal((70, 6))
    c = O.column_means(A)
    Ac = A - A.mean(axis=0)[None, :]
    assert np.allclose(O.apply_centred(A, X, c), Ac @ X, atol=1e-12)
    assert np.allclose(O.apply_centred_adjoint(A, Y, c), Ac.T @ Y, atol=1e-12)
    assert np.allclose(O.apply_centred(A, X, None), A @ X)
    assert np.allclose(O.apply_centred_adjoint(A, Y, None), A.T @ Y)


def test_exact_singular_values_matches_numpy():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((60, 25)) + 3.0
    for raw in (True, False):
        B = A if raw else A - A.mean(0)
        assert np.allclose(O.exact_singular_values(A, raw), np.linalg.svd(B, compute_uv=False), atol=1e-12)
    assert np.allclose(O.exact_singular_values(A.T, True), np.linalg.svd(A, compute_uv=False), atol=1e-12)


def test_normalise_signs():
    rng = np.random.default_rng(6)
    U = rng.standard_normal((10, 3))
    V = rng.standard_normal((7, 3))
    U2, V2 = O.normalise_signs(U, V)
    idx = np.argmax(np.abs(V2), axis=0)
    assert np.all(V2[idx, np.arange(3)] > 0)
    assert np.allclose(U2 @ V2.T, U @ V.T)

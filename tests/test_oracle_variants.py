"""Pins of the oracle's variants of the method (CPU, no GPU):

* Section 5's renormalisation schedule, and the odd-only schedule of its last
  paragraph, as step traces written out from the paper's description;
* odd-only renormalisation: same span as the full schedule (so the same result
  when the arithmetic has room), and the accuracy it gives up when a pair of
  unrenormalised products squares a dynamic range beyond the arithmetic;
* the self-adjoint loop (Section 5) with the two-sided projection: the full
  eigendecomposition at l = n, exact recovery of indefinite low-rank matrices,
  eigenvalue signs;
* the stabilised Nystrom method (Section 3): the Cholesky step against LAPACK,
  the closed form A_nu Q (Q^T A_nu Q)^-1 Q^T A_nu, exact recovery of
  nonnegative-definite low-rank matrices, and Section 3's claim that it is more
  accurate than the plain projection.
"""
import numpy as np
import pytest

import oracle as O
import synth as S


def _sym(n, lam, seed):
    Q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((n, n)))
    A = (Q * np.asarray(lam, dtype=np.float64)) @ Q.T
    return 0.5 * (A + A.T)


# ---------------------------------------------------------------------------
# renormalisation schedules
# ---------------------------------------------------------------------------

def test_general_schedule_trace():
    """Sketch, LU, then its x (A^*, LU, A, LU) with QR in place of the last LU, then
    the projection B^* = A^* Q (Sections 2 and 5)."""
    A = np.random.default_rng(0).standard_normal((50, 40))
    t = []
    O.rpca(A, 3, 5, 2, trace=t)
    assert t == ["A", "lu", "A*", "lu", "A", "lu", "A*", "lu", "A", "qr", "A*"]
    t = []
    O.rpca(A, 3, 5, 0, trace=t)
    assert t == ["A", "qr", "A*"]


def test_odd_only_schedule_trace():
    """Products numbered in order of application (sketch = 1); only the odd-numbered
    ones (the products with A) are renormalised; the final QR stays."""
    A = np.random.default_rng(0).standard_normal((50, 40))
    t = []
    O.rpca(A, 3, 5, 3, odd_only=True, trace=t)
    assert t == ["A", "lu", "A*", "A", "lu", "A*", "A", "lu", "A*", "A", "qr", "A*"]


def test_self_adjoint_loop_trace():
    """Section 5's printed loop with its = 4: A Q every iteration, LU when it < its,
    QR when it == its; odd-only drops the LU of the even iterations."""
    A = _sym(30, np.linspace(1, 0.1, 30), 1)
    t = []
    O.self_adjoint_range(A, 5, 4, trace=t)
    assert t == ["A", "lu", "A", "lu", "A", "lu", "A", "qr"]
    t = []
    O.self_adjoint_range(A, 5, 4, odd_only=True, trace=t)
    assert t == ["A", "lu", "A", "A", "lu", "A", "qr"]
    t = []
    O.rpca_sym(A, 3, 5, 1, trace=t)
    assert t == ["A", "qr", "A"]


def test_odd_only_keeps_the_span():
    """Every renormalisation multiplies by an invertible l x l matrix, so dropping some
    leaves the span, and the result, unchanged when nothing underflows the arithmetic."""
    sig = np.exp(-np.arange(1, 301) / 5.0)
    A = S.haar_dense_np(600, 300, sig, seed=3, dtype=np.float64)
    for its in (1, 2, 4):
        U, s, V = O.rpca(A, 10, 12, its, raw=True, seed=1)
        U2, s2, V2 = O.rpca(A, 10, 12, its, raw=True, seed=1, odd_only=True)
        assert np.max(np.abs(s - s2)) <= 1e-12 * s[0]
        assert np.linalg.norm(U.T @ U2 - np.diag(np.sign(np.diag(U.T @ U2))), 2) < 1e-8


def test_odd_only_loses_a_squared_dynamic_range():
    """With singular values from 1 down to 1e-11, an unrenormalised A (A^* Q) squares
    the range past FP64's 1e-16: the odd-only schedule loses sigma_9, sigma_10 while
    the full schedule keeps them to 1e-8 (the accuracy Section 5 says it sacrifices)."""
    sig = np.concatenate([10.0 ** -np.arange(0, 12, 1.0), np.full(288, 1e-13)])
    A = S.haar_dense_np(600, 300, sig, seed=3, dtype=np.float64)
    U, s, V = O.rpca(A, 10, 12, 2, raw=True, seed=1)
    U2, s2, V2 = O.rpca(A, 10, 12, 2, raw=True, seed=1, odd_only=True)
    full = np.abs(s - sig[:10]) / sig[:10]
    odd = np.abs(s2 - sig[:10]) / sig[:10]
    assert full.max() < 1e-8
    assert odd[:6].max() < 1e-10 and odd[8:].min() > 0.1


# ---------------------------------------------------------------------------
# self-adjoint A
# ---------------------------------------------------------------------------

def test_sym_full_width_is_the_eigendecomposition():
    n = 40
    lam = np.concatenate([np.linspace(3, 1, 20), -np.linspace(2.5, 0.1, 20)])
    A = _sym(n, lam, 4)
    U, s, V = O.rpca_sym(A, n, n, 2, seed=2)
    assert np.allclose((U * s) @ V.T, A, atol=1e-11 * np.abs(lam).max())
    ev = np.linalg.eigvalsh(A)
    order = np.argsort(-np.abs(ev), kind="stable")
    assert np.allclose(s, np.abs(ev[order]), rtol=1e-12, atol=1e-13)
    # V = U diag(sign(lambda)): U^T V is diagonal with the eigenvalue signs
    D = U.T @ V
    assert np.allclose(D, np.diag(np.sign(ev[order])), atol=1e-10)


@pytest.mark.parametrize("its", [1, 2, 3])
def test_sym_exact_low_rank_recovery(its):
    n, r = 200, 6
    lam = np.concatenate([[4.0, -3.0, 2.0, -1.5, 1.0, 0.5], np.zeros(n - r)])
    A = _sym(n, lam, 9)
    U, s, V = O.rpca_sym(A, r, r + 2, its, seed=5)
    E = A - (U * s) @ V.T
    assert np.linalg.norm(E, 2) <= 1e-12 * np.linalg.norm(A, 2)
    assert np.allclose(s, np.sort(np.abs(lam[:r]))[::-1], rtol=1e-12)


def test_sym_residual_approaches_best():
    lam = (-1.0) ** np.arange(300) / np.arange(1, 301)
    A = _sym(300, lam, 2)
    best = 1.0 / 11
    errs = []
    for its in (1, 3, 6):
        U, s, V = O.rpca_sym(A, 10, 12, its, seed=3)
        errs.append(np.linalg.norm(A - (U * s) @ V.T, 2))
    assert errs[0] >= best * (1 - 1e-12) and errs[2] <= errs[0] and errs[2] <= 1.5 * best


# ---------------------------------------------------------------------------
# the stabilised Nystrom method (Section 3)
# ---------------------------------------------------------------------------

def test_cholesky_upper_matches_lapack():
    B = np.random.default_rng(3).standard_normal((25, 25))
    B = B @ B.T + 25 * np.eye(25)
    C = O.cholesky_upper(B)
    assert np.allclose(C, np.linalg.cholesky(B).T, rtol=1e-13, atol=1e-13)
    assert np.allclose(np.tril(C, -1), 0.0)


def test_nystrom_closed_form_with_the_shift():
    """With k = l nothing is truncated or clipped: U diag(Sigma + nu) U^T equals the
    Nystrom approximation A_nu Q (Q^T A_nu Q)^-1 Q^T A_nu of A_nu = A + nu I."""
    n, l = 120, 10
    A = _sym(n, 1.0 / np.arange(1, n + 1) ** 2, 6)
    U, Sg = O.nystrom(A, l, l, 2, seed=4)
    Q = O.self_adjoint_range(A, l, 2, seed=4)
    nu = O.nystrom_shift(Q.T @ A @ Q, n)
    Anu = A + nu * np.eye(n)
    ref = Anu @ Q @ np.linalg.solve(Q.T @ Anu @ Q, Q.T @ Anu)
    assert np.allclose((U * (Sg + nu)) @ U.T, ref, atol=1e-12)


def test_nystrom_exact_low_rank_recovery():
    n, r = 150, 5
    A = _sym(n, np.concatenate([[5.0, 3.0, 2.0, 1.0, 0.25], np.zeros(n - r)]), 8)
    U, Sg = O.nystrom(A, r, r + 3, 1, seed=1)
    assert np.linalg.norm(A - (U * Sg) @ U.T, 2) <= 1e-9 * 5.0
    assert np.allclose(Sg, [5.0, 3.0, 2.0, 1.0, 0.25], rtol=1e-9)


@pytest.mark.parametrize("seed", range(5))
def test_nystrom_more_accurate_than_projection(seed):
    """Section 3: for nonnegative-definite A the Nystrom approximation beats the
    approximation of Eqs. i2-i4 built from the same Q (slowly decaying spectrum)."""
    n = 300
    A = _sym(n, 1.0 / np.arange(1, n + 1), seed)
    U, Sg = O.nystrom(A, 10, 12, 1, seed=seed)
    Us, Ss, Vs = O.rpca_sym(A, 10, 12, 1, seed=seed)
    e_nys = np.linalg.norm(A - (U * Sg) @ U.T, 2)
    e_proj = np.linalg.norm(A - (Us * Ss) @ Vs.T, 2)
    assert e_nys < e_proj
    assert e_nys >= (1.0 / 11) * (1 - 1e-12)       # Eckart-Young

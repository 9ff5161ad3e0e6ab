"""Plain FP64 CPU oracle for the randomized PCA of Szlam, Kluger & Tygert (2014).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module.  The CUDA library never calls it and shares no code with it.

Everything is written for a reader checking it against the paper by eye: the
steps follow the paper's order and notation, in FP64, with a matrix product
(numpy ``@``) as the only library primitive used by the method itself.  There
is no blocking, fusion or reordering beyond what the paper states.

Sections and equations cited:

* Section 2 (Overview), Eqs. (i1)-(approx): Q with orthonormal columns nearly
  spanning range(A); B = Q^* A (i2); W Sigma V^* = B (i3); U = Q W (i4).
  Random test vectors with i.i.d. N(0,1) entries; power iterations applying
  A and A^* alternately; renormalisation after every application.
* Section 5 (Algorithmic optimizations): LU renormalisation ([Q,R] = lu(Q),
  MATLAB's two-output form, so Q = P^T L) after every product but the last,
  which is an (unpivoted) economy QR; implicit centring
  A*Q - ones(m,1)*(c*Q) with c the row vector of column means; the adjoint
  applied as (Q'*A)'.
* Section 4 (Measuring accuracy): the spectral norm of A - U Sigma V^*
  estimated by the power method from a random start.
* Section 5, self-adjoint A: the printed loop Q = A*Q with LU on all but the
  last iteration and QR on the last (``self_adjoint_range``, ``rpca_sym``);
  the last paragraph's renormalisation in odd-numbered iterations only
  (``odd_only``).
* Section 3 (Stabilizing the Nystrom method): B1 = A Q, B2 = Q^* B1,
  C^* C = B2, F = B1 C^-1, U S V^* = F, Sigma = S^2, stabilised by adding a
  multiple of the identity and subtracting it again (``nystrom``).

The Gaussian test matrix is drawn from Philox4x64-10 (Salmon, Moraes, Dror &
Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11) with the
Box-Muller transform, keyed by (seed, stream) with counter = block index; the
CUDA side implements the same published generator independently.

Parity pins (tests/test_oracle_*.py): numpy's own Philox bit generator,
scipy's LU, numpy's QR and SVD, explicit centring, exact recovery of exactly
low-rank matrices, the worked examples of Section 6, the Eckart-Young lower
bound and the factor-of-two claims of Sections 7-8.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "philox4x64_10", "uniform23", "gaussian_omega", "column_means",
    "apply_centred", "apply_centred_adjoint", "lu_renorm", "householder_qr",
    "jacobi_svd", "round_robin_steps", "normalise_signs", "rpca",
    "self_adjoint_range", "rpca_sym", "cholesky_upper", "nystrom_shift", "nystrom",
    "resid_power", "resid_exact", "exact_singular_values",
]

_MASK64 = (1 << 64) - 1
_U32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)

# Philox4x64 multipliers and Weyl key increments (SC'11, Section 4).
PHILOX_M0 = 0xD2E7470EE14C6C93
PHILOX_M1 = 0xCA5A826395121157
PHILOX_W0 = 0x9E3779B97F4A7C15
PHILOX_W1 = 0xBB67AE8584CAA73B


def _mulhilo64(a: int, b: np.ndarray):
    """(hi, lo) 64-bit halves of the 128-bit product of the constant a and each b."""
    a_lo = np.uint64(a & 0xFFFFFFFF)
    a_hi = np.uint64(a >> 32)
    b_lo = b & _U32
    b_hi = b >> _S32
    ll = a_lo * b_lo
    lh = a_lo * b_hi
    hl = a_hi * b_lo
    hh = a_hi * b_hi
    mid = (ll >> _S32) + (lh & _U32) + (hl & _U32)
    lo = (ll & _U32) | ((mid & _U32) << _S32)
    hi = hh + (lh >> _S32) + (hl >> _S32) + (mid >> _S32)
    return hi, lo


def philox4x64_10(counters: np.ndarray, key0: int, key1: int) -> np.ndarray:
    """Philox4x64 with 10 rounds.  counters: uint64 array (N, 4); returns (N, 4).

    One round maps (x0, x1, x2, x3) with key (k0, k1) to
    (hi(M1*x2) ^ x1 ^ k0, lo(M1*x2), hi(M0*x0) ^ x3 ^ k1, lo(M0*x0)); the key
    is bumped by the Weyl constants (W0, W1) before every round but the first.
    """
    x = [np.array(counters[:, i], dtype=np.uint64) for i in range(4)]
    k0, k1 = key0 & _MASK64, key1 & _MASK64
    with np.errstate(over="ignore"):
        for r in range(10):
            if r > 0:
                k0 = (k0 + PHILOX_W0) & _MASK64
                k1 = (k1 + PHILOX_W1) & _MASK64
            hi0, lo0 = _mulhilo64(PHILOX_M0, x[0])
            hi1, lo1 = _mulhilo64(PHILOX_M1, x[2])
            x = [hi1 ^ x[1] ^ np.uint64(k0), lo1, hi0 ^ x[3] ^ np.uint64(k1), lo0]
    return np.stack(x, axis=1)


def uniform23(bits: np.ndarray) -> np.ndarray:
    """Top 23 bits b of a 64-bit word mapped to the open interval (0, 1): (b + 1/2) / 2^23.

    Every such value has at most 24 significant bits, so it is exact in FP32
    as well as FP64: both implementations start Box-Muller from the same u.
    """
    return ((bits >> np.uint64(41)).astype(np.float64) + 0.5) * (2.0 ** -23)


def gaussian_omega(n: int, l: int, seed: int, stream: int = 0) -> np.ndarray:
    """n x l matrix of i.i.d. N(0,1) draws (Section 2; Section 5 allows any i.i.d. law).

    Entry (i, j) is element e = i*l + j of a stream in which Philox block b
    (counter (b, 0, 0, 0), key (seed, stream)) gives four words w0..w3 that
    Box-Muller turns into elements 4b..4b+3:
    sqrt(-2 ln u0) cos(2 pi u1), sqrt(-2 ln u0) sin(2 pi u1), and likewise
    for (u2, u3), with u = uniform23(w).
    """
    total = n * l
    nblk = (total + 3) // 4
    ctr = np.zeros((nblk, 4), dtype=np.uint64)
    ctr[:, 0] = np.arange(nblk, dtype=np.uint64)
    w = philox4x64_10(ctr, seed, stream)
    u = uniform23(w)
    r0 = np.sqrt(-2.0 * np.log(u[:, 0]))
    r1 = np.sqrt(-2.0 * np.log(u[:, 2]))
    z = np.empty((nblk, 4))
    z[:, 0] = r0 * np.cos(2.0 * np.pi * u[:, 1])
    z[:, 1] = r0 * np.sin(2.0 * np.pi * u[:, 1])
    z[:, 2] = r1 * np.cos(2.0 * np.pi * u[:, 3])
    z[:, 3] = r1 * np.sin(2.0 * np.pi * u[:, 3])
    return z.reshape(-1)[:total].reshape(n, l)


# ---------------------------------------------------------------------------
# implicit centring (Section 5)
# ---------------------------------------------------------------------------

def _as_f64(A):
    """A widened to FP64; a scipy sparse matrix stays sparse (Section 5: the same code
    serves dense and sparse A, through products only)."""
    import scipy.sparse as sp
    if sp.issparse(A):
        return sp.csr_matrix(A, dtype=np.float64)
    return np.asarray(A, dtype=np.float64)


def column_means(A) -> np.ndarray:
    """c: the 1 x n vector of the means of the columns of A (Section 5)."""
    return np.asarray(_as_f64(A).mean(axis=0), dtype=np.float64).ravel()


def apply_centred(A, X, c):
    """A_c X = A*X - ones(m,1)*(c*X): the mean-centred A applied without forming it.

    ``c`` is None when the matrix is used raw (no centring).
    """
    Y = np.asarray(A @ X)
    if c is not None:
        Y = Y - np.ones((A.shape[0], 1)) @ (c[None, :] @ X)
    return Y


def apply_centred_adjoint(A, Y, c):
    """A_c^* Y = (Y'*A)' - c' * (ones(1,m)*Y): the adjoint applied through A itself."""
    X = np.asarray(Y.T @ A).T
    if c is not None:
        X = X - c[:, None] @ (np.ones((1, A.shape[0])) @ Y)
    return X


# ---------------------------------------------------------------------------
# renormalisations (Section 5)
# ---------------------------------------------------------------------------

def lu_renorm(Y: np.ndarray):
    """MATLAB's two-output ``[Q, R] = lu(Y)`` for a tall m x l matrix.

    Gaussian elimination with partial pivoting: at column j the row of largest
    |entry| at or below the diagonal (the first one on ties) becomes the pivot.
    Returns (Q, R) with Q = P^T L (m x l, a row permutation of a unit
    lower-trapezoidal L with |L| <= 1) and R upper triangular (l x l), such
    that Q R = Y.  A zero pivot leaves its column unscaled, as LAPACK does.
    """
    W = np.array(Y, dtype=np.float64, copy=True)
    m, l = W.shape
    perm = np.arange(m)
    for j in range(min(m, l)):
        p = j + int(np.argmax(np.abs(W[j:, j])))
        if p != j:
            W[[j, p], :] = W[[p, j], :]
            perm[[j, p]] = perm[[p, j]]
        piv = W[j, j]
        if piv != 0.0:
            W[j + 1:, j] /= piv
            W[j + 1:, j + 1:] -= np.outer(W[j + 1:, j], W[j, j + 1:])
    L = np.tril(W[:, :l], -1)
    L[np.arange(min(m, l)), np.arange(min(m, l))] = 1.0
    R = np.triu(W[:l, :])
    Q = np.empty_like(L)
    Q[perm] = L
    return Q, R


def householder_qr(Y: np.ndarray):
    """Economy QR by Householder reflections (``[Q, R] = qr(Y, 0)``, unpivoted).

    Returns Q (m x l, orthonormal columns) and R (l x l, upper triangular).
    """
    R = np.array(Y, dtype=np.float64, copy=True)
    m, l = R.shape
    vs = []
    for j in range(l):
        x = R[j:, j]
        nx = np.linalg.norm(x)
        v = x.copy()
        v[0] += (1.0 if x[0] >= 0 else -1.0) * nx
        nv = np.linalg.norm(v)
        if nv == 0.0:
            vs.append(None)
            continue
        v /= nv
        R[j:, j:] -= 2.0 * np.outer(v, v @ R[j:, j:])
        vs.append(v)
    Q = np.eye(m, l)
    for j in range(l - 1, -1, -1):
        v = vs[j]
        if v is not None:
            Q[j:, :] -= 2.0 * np.outer(v, v @ Q[j:, :])
    return Q, np.triu(R[:l, :])


# ---------------------------------------------------------------------------
# one-sided Jacobi SVD (Hestenes; Golub & Van Loan Sec. 8.6; Demmel & Veselic 1992)
# ---------------------------------------------------------------------------

def round_robin_steps(q: int):
    """Brent-Luk round-robin ordering: q-1 (q even) steps of q/2 disjoint column pairs."""
    qq = q + (q % 2)
    arr = list(range(qq))
    steps = []
    for _ in range(qq - 1):
        ps, qs = [], []
        for i in range(qq // 2):
            a, b = arr[i], arr[qq - 1 - i]
            if a < q and b < q:
                ps.append(min(a, b))
                qs.append(max(a, b))
        steps.append((np.array(ps, dtype=np.int64), np.array(qs, dtype=np.int64)))
        arr = [arr[0]] + [arr[-1]] + arr[1:-1]
    return steps


def jacobi_svd(M: np.ndarray, tol: float | None = None, max_sweeps: int = 80):
    """Full SVD M = U diag(s) V^T by one-sided Jacobi rotations, FP64.

    For a tall (or square) M the columns are orthogonalised by plane rotations
    applied on the right until every pair (p, q) satisfies
    |m_p . m_q| <= tol * |m_p| |m_q|; then s_j = |m_j|, U_j = m_j / s_j and V
    is the product of the rotations.  A wide M is handled through M^T.
    Singular values are returned in descending order.  Columns of U whose
    singular value is negligible are completed to an orthonormal set.
    """
    M = np.asarray(M, dtype=np.float64)
    p, q = M.shape
    if p < q:
        U, s, V = jacobi_svd(M.T, tol, max_sweeps)
        return V, s, U
    if tol is None:
        tol = max(p, q) * np.finfo(np.float64).eps
    W = M.copy()
    J = np.eye(q)
    steps = round_robin_steps(q)
    for _ in range(max_sweeps):
        rotated = False
        for P, Qc in steps:
            if P.size == 0:
                continue
            a = W[:, P]
            b = W[:, Qc]
            alpha = np.einsum("ij,ij->j", a, a)
            beta = np.einsum("ij,ij->j", b, b)
            gamma = np.einsum("ij,ij->j", a, b)
            act = np.abs(gamma) > tol * np.sqrt(alpha * beta)
            if not act.any():
                continue
            rotated = True
            g = np.where(act, gamma, 1.0)
            zeta = (beta - alpha) / (2.0 * g)
            t = np.where(zeta >= 0, 1.0, -1.0) / (np.abs(zeta) + np.sqrt(1.0 + zeta * zeta))
            cs = 1.0 / np.sqrt(1.0 + t * t)
            sn = cs * t
            cs = np.where(act, cs, 1.0)
            sn = np.where(act, sn, 0.0)
            W[:, P] = cs * a - sn * b
            W[:, Qc] = sn * a + cs * b
            ja = J[:, P]
            jb = J[:, Qc]
            J[:, P] = cs * ja - sn * jb
            J[:, Qc] = sn * ja + cs * jb
        if not rotated:
            break
    s = np.linalg.norm(W, axis=0)
    order = np.argsort(-s, kind="stable")
    s = s[order]
    W = W[:, order]
    J = J[:, order]
    U = np.zeros_like(W)
    smax = s[0] if s.size else 0.0
    small = s <= max(p, q) * np.finfo(np.float64).eps * smax
    U[:, ~small] = W[:, ~small] / s[~small]
    for j in np.nonzero(small)[0]:          # orthonormal completion for null directions
        for e in range(p):
            v = np.zeros(p)
            v[e] = 1.0
            for _ in range(2):
                v -= U[:, :j] @ (U[:, :j].T @ v)
                v -= U[:, j + 1:] @ (U[:, j + 1:].T @ v)
            nv = np.linalg.norm(v)
            if nv > 0.5:
                U[:, j] = v / nv
                break
    return U, s, J


def normalise_signs(U: np.ndarray, V: np.ndarray):
    """Flip each (U_j, V_j) pair so that the entry of V_j of largest magnitude is positive.

    The paper leaves the sign of singular vectors free; this fixes one.  Ties
    go to the first (lowest-index) entry.
    """
    U = U.copy()
    V = V.copy()
    idx = np.argmax(np.abs(V), axis=0)
    flip = V[idx, np.arange(V.shape[1])] < 0
    U[:, flip] *= -1.0
    V[:, flip] *= -1.0
    return U, V


# ---------------------------------------------------------------------------
# the method (Sections 2 and 5)
# ---------------------------------------------------------------------------

def rpca(A, k: int, l: int | None = None, its: int = 2, raw: bool = False,
         seed: int = 0, omega: np.ndarray | None = None, odd_only: bool = False,
         trace: list | None = None):
    """Rank-k approximation A_c ~ U diag(S) V^T by the randomized method.

    A: m x n (any real dtype; widened to FP64).  l defaults to k + 2 and its
    to 2, the paper's defaults.  With raw=False the column means are removed
    implicitly (Section 5).  Steps:

    1. Y = A_c Omega, Omega n x l i.i.d. N(0,1) (Section 2).
    2. its = 0: Q = qr(Y).  Otherwise Q = lu(Y), then for it = 1..its:
       Q = lu(A_c^* Q); Y = A_c Q; Q = lu(Y) if it < its else qr(Y)
       (Section 5: LU after every application but the last, which is QR).
    3. B = Q^* A_c, computed as (A_c^* Q)^* (Eq. i2; Section 5's adjoint).
    4. W Sigma V^* = B by one-sided Jacobi (Eq. i3); U = Q W (Eq. i4).
    5. Keep the leading k triplets; fix signs as in ``normalise_signs``.
    Returns (U m x k, S k, V n x k), all FP64.

    odd_only: Section 5's last optimisation, renormalising only after the
    odd-numbered applications.  The products are numbered in the order they
    are applied (the sketch is the first, then A^* and A alternate), as the
    self-adjoint loop of Section 5 numbers its one product per iteration; so
    the LU after every product with A^* is dropped and the pair A_c (A_c^* Q)
    is applied unrenormalised.  The final QR is kept.
    trace: when a list is given, the steps are appended to it by name
    ("A", "A*", "lu", "qr"), for checking the control flow.
    """
    A = _as_f64(A)
    m, n = A.shape
    if l is None:
        l = k + 2
    if not (1 <= k <= l <= min(m, n)) or its < 0:
        raise ValueError("need 1 <= k <= l <= min(m, n) and its >= 0")
    log = trace.append if trace is not None else (lambda _s: None)
    c = None if raw else column_means(A)
    Om = gaussian_omega(n, l, seed) if omega is None else np.asarray(omega, dtype=np.float64)
    Y = apply_centred(A, Om, c)
    log("A")
    if its == 0:
        Q, _ = householder_qr(Y)
        log("qr")
    else:
        Q, _ = lu_renorm(Y)
        log("lu")
        for it in range(1, its + 1):
            Q = apply_centred_adjoint(A, Q, c)
            log("A*")
            if not odd_only:
                Q, _ = lu_renorm(Q)
                log("lu")
            Y = apply_centred(A, Q, c)
            log("A")
            Q, _ = lu_renorm(Y) if it < its else householder_qr(Y)
            log("lu" if it < its else "qr")
    Bt = apply_centred_adjoint(A, Q, c)      # n x l, = B^*
    log("A*")
    W, s, V = jacobi_svd(Bt.T)               # B = W diag(s) V^T
    U = Q @ W[:, :k]
    U, V = normalise_signs(U, V[:, :k])
    return U, s[:k].copy(), V


# ---------------------------------------------------------------------------
# self-adjoint A (Section 5's loop) and the stabilised Nystrom method (Section 3)
# ---------------------------------------------------------------------------

def self_adjoint_range(A, l: int, its: int, seed: int = 0, omega: np.ndarray | None = None,
                       odd_only: bool = False, trace: list | None = None) -> np.ndarray:
    """Section 5's core iterations for a self-adjoint n x n A, as printed there.

    Q starts as the n x l random matrix (Section 2).  For it = 1..its:
    Q = A Q; then Q = lu(Q) when it < its, and Q = qr(Q) when it == its.
    With odd_only (Section 5's last paragraph) the LU runs only when it is odd.
    Returns the n x l orthonormal Q.  Needs its >= 1 (with none, Q would be the
    random matrix itself).
    """
    A = _as_f64(A)
    n = A.shape[0]
    if A.shape[1] != n or its < 1 or not (1 <= l <= n):
        raise ValueError("need a square A, its >= 1 and 1 <= l <= n")
    log = trace.append if trace is not None else (lambda _s: None)
    Q = gaussian_omega(n, l, seed) if omega is None else np.asarray(omega, dtype=np.float64)
    for it in range(1, its + 1):
        Q = np.asarray(A @ Q)
        log("A")
        if it < its and (not odd_only or it % 2 == 1):
            Q, _ = lu_renorm(Q)
            log("lu")
        if it == its:
            Q, _ = householder_qr(Q)
            log("qr")
    return Q


def rpca_sym(A, k: int, l: int | None = None, its: int = 2, seed: int = 0,
             omega: np.ndarray | None = None, odd_only: bool = False, trace: list | None = None):
    """Rank-k approximation of a self-adjoint A (n x n): A ~ U diag(S) V^T with
    V = U diag(sign(lambda)), i.e. A ~ U diag(lambda) U^T.

    1. Q from ``self_adjoint_range`` (only products with A: A^* = A).
    2. B = Q^* A Q (l x l), symmetrised as (B + B^T) / 2 (the projection of
       Eq. i2 taken on both sides, which keeps the approximation self-adjoint).
    3. B = W diag(s) J^T by one-sided Jacobi (Eq. i3); for symmetric B,
       J_j = sign(lambda_j) W_j, so lambda_j = s_j sign(W_j . J_j).
    4. U = Q W, V = Q J (Eq. i4), leading k; signs as in ``normalise_signs``.
    The column centring of Section 5 does not apply: the centred matrix of a
    self-adjoint A is not self-adjoint.  Returns (U, S, V), FP64.
    """
    A = _as_f64(A)
    n = A.shape[0]
    if l is None:
        l = k + 2
    if not (1 <= k <= l <= n):
        raise ValueError("need 1 <= k <= l <= n")
    log = trace.append if trace is not None else (lambda _s: None)
    Q = self_adjoint_range(A, l, its, seed, omega, odd_only, trace)
    Z = np.asarray(A @ Q)
    log("A")
    B = Q.T @ Z
    B = 0.5 * (B + B.T)
    W, s, J = jacobi_svd(B)
    U, V = normalise_signs(Q @ W[:, :k], Q @ J[:, :k])
    return U, s[:k].copy(), V


def cholesky_upper(B: np.ndarray) -> np.ndarray:
    """Upper-triangular C with C^T C = B for a symmetric positive-definite B (the
    textbook column-by-column Cholesky): C_jj = sqrt(B_jj - sum_{t<j} C_tj^2),
    C_ji = (B_ji - sum_{t<j} C_tj C_ti) / C_jj for i > j."""
    B = np.asarray(B, dtype=np.float64)
    l = B.shape[0]
    C = np.zeros_like(B)
    for j in range(l):
        d = B[j, j] - C[:j, j] @ C[:j, j]
        if not d > 0.0:
            raise np.linalg.LinAlgError("matrix is not positive definite")
        C[j, j] = math.sqrt(d)
        C[j, j + 1:] = (B[j, j + 1:] - C[:j, j] @ C[:j, j + 1:]) / C[j, j]
    return C


# Unit roundoff of the FP32 arithmetic the shift of the Nystrom method is scaled by.
NYSTROM_U = 2.0 ** -24


def nystrom_shift(B2: np.ndarray, n: int) -> float:
    """The multiple nu of the identity added to A (and subtracted from the result).

    Section 3 leaves its size open ("an appropriate multiple"); the reading
    taken is nu = 2 (16 l + sqrt(n)) u tr(B2) with u = 2^-24 and B2 = Q^* A Q
    (l x l): twice the sum of the pivot size below which an FP32 Cholesky of
    an l x l matrix is taken to have collapsed (16 l u of a diagonal entry)
    and the FP32 rounding of the n-term products that form B2 (about
    sqrt(n) u |A| per entry), relative to tr(B2) >= |B2|.  Then B2 + nu I is
    safely positive definite in FP32 arithmetic.
    """
    l = B2.shape[0]
    return 2.0 * (16.0 * l + math.sqrt(n)) * NYSTROM_U * float(np.trace(B2))


def nystrom(A, k: int, l: int | None = None, its: int = 2, seed: int = 0,
            omega: np.ndarray | None = None, odd_only: bool = False):
    """Stabilised Nystrom approximation A ~ U diag(S) U^T of a self-adjoint,
    nonnegative-definite A (n x n), Section 3 with the identity shift.

    Q: the orthonormal n x l basis of ``self_adjoint_range``.  Then, for
    A + nu I (nu from ``nystrom_shift`` of Q^* A Q):
      B1 = A Q + nu Q                  (eq. start)
      B2 = Q^* B1, symmetrised         (eq. second)
      C^* C = B2, C upper triangular   (eq. Cholesky)
      F = B1 C^-1                      (eq. pseudo, by triangular solves)
      U S V^* = F                      (one-sided Jacobi on F)
      Sigma = S^2 - nu, clipped at 0   (eq. finish, the shift subtracted)
    Returns (U n x k, Sigma k), leading k, each U column's largest-|entry|
    positive, FP64.
    """
    A = _as_f64(A)
    n = A.shape[0]
    if l is None:
        l = k + 2
    if not (1 <= k <= l <= n):
        raise ValueError("need 1 <= k <= l <= n")
    Q = self_adjoint_range(A, l, its, seed, omega, odd_only)
    AQ = np.asarray(A @ Q)
    B2 = Q.T @ AQ
    nu = nystrom_shift(0.5 * (B2 + B2.T), n)
    B1 = AQ + nu * Q
    B2 = Q.T @ B1
    B2 = 0.5 * (B2 + B2.T)
    C = cholesky_upper(B2)                  # C^* C = B2, C upper triangular
    # F C = B1 by forward substitution on the columns of F (C upper triangular)
    F = np.zeros_like(B1)
    for j in range(l):
        F[:, j] = (B1[:, j] - F[:, :j] @ C[:j, j]) / C[j, j]
    Uf, s, _ = jacobi_svd(F)
    U = Uf[:, :k]
    idx = np.argmax(np.abs(U), axis=0)
    U = U * np.where(U[idx, np.arange(k)] < 0, -1.0, 1.0)[None, :]
    return U, np.maximum(s[:k] ** 2 - nu, 0.0)


# ---------------------------------------------------------------------------
# accuracy (Section 4)
# ---------------------------------------------------------------------------

def resid_power(A, U, S, V, raw: bool = False, iters: int = 20, seed: int = 0):
    """Power-method estimate of ||A_c - U diag(S) V^T|| from a random start (Section 4).

    x_0: N(0,1) n-vector from the Philox stream (seed, 1), normalised.  Each
    iteration forms z = E^T (E x) with E applied implicitly (centring as in
    Section 5, the approximation as U (S (V^T x))), takes lambda = |z| and
    x = z / |z|.  Returns sqrt(lambda) after ``iters`` iterations; since
    |E^T E x| <= ||E||^2 for unit x the estimate never exceeds ||E||.
    """
    A = _as_f64(A)
    U = np.asarray(U, dtype=np.float64)
    S = np.asarray(S, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    c = None if raw else column_means(A)
    x = gaussian_omega(A.shape[1], 1, seed, stream=1)
    x /= np.linalg.norm(x)
    lam = 0.0
    for _ in range(iters):
        y = apply_centred(A, x, c) - U @ (S[:, None] * (V.T @ x))
        z = apply_centred_adjoint(A, y, c) - V @ (S[:, None] * (U.T @ y))
        lam = float(np.linalg.norm(z))
        if lam == 0.0:
            return 0.0
        x = z / lam
    return math.sqrt(lam)


def resid_exact(A, U, S, V, raw: bool = False) -> float:
    """||A_c - U diag(S) V^T||_2 from the full Jacobi SVD of the dense residual (small sizes)."""
    A = _as_f64(A)
    A = A.toarray() if hasattr(A, "toarray") else A
    E = A - (0.0 if raw else column_means(A)[None, :]) - (np.asarray(U) * np.asarray(S)[None, :]) @ np.asarray(V).T
    return float(jacobi_svd(E)[1][0])


def exact_singular_values(A, raw: bool = False) -> np.ndarray:
    """All singular values of A_c, descending, from the FP64 Gram of the narrower side.

    Used as ground truth for sigma_{k+1}.  Squaring costs relative accuracy
    u * (sigma_1 / sigma_j)^2 in FP64, i.e. 1e-10 at sigma_j = 1e-3 sigma_1.
    """
    A = _as_f64(A)
    A = A.toarray() if hasattr(A, "toarray") else A
    if not raw:
        A = A - A.mean(axis=0)[None, :]
    G = A.T @ A if A.shape[0] >= A.shape[1] else A @ A.T
    ev = np.linalg.eigvalsh(G)[::-1]
    return np.sqrt(np.clip(ev, 0.0, None))

"""Pins for the oracle's whole method (Sections 2, 4, 5, 6, 7) against facts the
paper and the mathematics fix: exact recovery of low-rank matrices, the full
SVD when l = min(m, n), the worked examples of Section 6, the Eckart-Young
bound and the near-optimal accuracy claims of Section 7, and the properties of
the power-method residual estimator (Section 4).
"""
import json
import os

import numpy as np
import pytest

import oracle as O
import synth as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _lowrank(m, n, r, seed, offset=0.0):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((m, r)) @ rng.standard_normal((r, n)) + offset


@pytest.mark.parametrize("raw", [True, False])
@pytest.mark.parametrize("its", [0, 1, 2])
def test_exact_recovery_of_low_rank(raw, its):
    # rank r <= l (centring adds at most one to the rank of A - 1 c)
    r = 8 if raw else 7
    A = _lowrank(120, 90, r, 11 + its, offset=0.0 if raw else 3.0)
    U, S_, V = O.rpca(A, k=8, l=10, its=its, raw=raw, seed=3)
    Ac = A if raw else A - A.mean(0)
    err = np.linalg.norm(Ac - (U * S_) @ V.T, 2) / np.linalg.norm(Ac, 2)
    assert err < 1e-12


@pytest.mark.parametrize("raw", [True, False])
def test_full_width_sketch_gives_truncated_svd(raw):
    rng = np.random.default_rng(21)
    A = rng.standard_normal((80, 30)) + (0.0 if raw else 2.0)
    Ac = A if raw else A - A.mean(0)
    Un, sn, Vtn = np.linalg.svd(Ac, full_matrices=False)
    U, S_, V = O.rpca(A, k=12, l=30, its=0, raw=raw, seed=4)
    assert np.allclose(S_, sn[:12], rtol=1e-12)
    assert np.allclose(U @ U.T, Un[:, :12] @ Un[:, :12].T, atol=1e-11)
    assert np.allclose(V @ V.T, Vtn[:12].T @ Vtn[:12], atol=1e-11)
    assert np.allclose(U.T @ U, np.eye(12), atol=1e-12)


def test_section6_worked_examples():
    with open(os.path.join(GOLDEN, "section6_lanczos_failures.json")) as f:
        gold = json.load(f)
    for case in gold["cases"]:
        A = S.propack_diag(case["size"])
        k = case["k"]
        _, S_, _ = O.rpca(A, k=k, l=k + 2, its=2, raw=True, seed=17)
        assert np.allclose(S_, np.array(case["expect_sorted"], dtype=np.float64), atol=1e-7, rtol=0)


def test_section7_spectra_eckart_young_and_near_optimal():
    with open(os.path.join(GOLDEN, "section7_spectra.json")) as f:
        gold = json.load(f)
    st = gold["settings"][0]
    m, n, k = st["m"], st["n"], st["k"]
    best = gold["best_rank_k_error"]
    for kind in gold["kinds"]:
        sig = S.spectrum_section7(kind, k, min(m, n))
        assert np.isclose(sig.max(), gold["spectral_norm"])
        assert np.isclose(np.sort(sig)[::-1][k], best)
        A = S.haar_dense_np(m, n, sig, seed=100 + kind, dtype=np.float64)
        for dl in (2, 8):
            U, S_, V = O.rpca(A, k=k, l=k + dl, its=2, raw=True, seed=kind * 10 + dl)
            e = np.linalg.norm(A - (U * S_) @ V.T, 2)
            assert e >= best * (1 - 1e-6)        # no rank-k approximation beats sigma_{k+1}
            assert e <= 2.0 * best               # "never greater than twice the best"
            assert np.isclose(O.resid_exact(A, U, S_, V, raw=True), e, rtol=1e-10)


def test_more_power_iterations_approach_optimal():
    # Section 7 second experiment: mean sqrt(30/n) Gaussian with sign flips; its = 0 is
    # far from optimal, its = 2 and 4 nearly optimal; the best error is about ||A|| / 2.
    n, k = 300, 4
    A = S.e2_matrix_np(n, seed=7).astype(np.float64)
    s = np.linalg.svd(A, compute_uv=False)
    best = s[k]
    assert 0.35 < best / s[0] < 0.65
    errs = {}
    for its in (0, 2, 4, 8):
        e = []
        for t in range(5):
            U, S_, V = O.rpca(A, k=k, l=k + 2, its=its, raw=True, seed=1000 * its + t)
            e.append(np.linalg.norm(A - (U * S_) @ V.T, 2))
        errs[its] = np.mean(e)
    assert errs[0] > 1.15 * best
    assert errs[2] < 1.1 * best and errs[4] < 1.05 * best and errs[8] < 1.03 * best
    assert errs[8] <= errs[2] * 1.001


def test_centring_equals_raw_on_explicitly_centred():
    rng = np.random.default_rng(31)
    A = rng.standard_normal((150, 60)) @ np.diag(np.linspace(3, 0.1, 60)) + 4.0
    Om = O.gaussian_omega(60, 9, seed=2)
    U1, S1, V1 = O.rpca(A, k=7, l=9, its=2, raw=False, omega=Om)
    U2, S2, V2 = O.rpca(A - A.mean(0), k=7, l=9, its=2, raw=True, omega=Om)
    assert np.allclose(S1, S2, rtol=1e-10)
    assert np.allclose(U1, U2, atol=1e-8) and np.allclose(V1, V2, atol=1e-8)


def test_seed_and_omega_agree():
    A = _lowrank(50, 40, 12, 3) + 0.01 * np.random.default_rng(1).standard_normal((50, 40))
    a = O.rpca(A, k=5, l=8, its=1, raw=False, seed=9)
    b = O.rpca(A, k=5, l=8, its=1, raw=False, omega=O.gaussian_omega(40, 8, 9))
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("raw", [True, False])
def test_residual_estimator_bounds(raw):
    rng = np.random.default_rng(41)
    A = (rng.standard_normal((90, 70)) @ np.diag(0.8 ** np.arange(70)) @ rng.standard_normal((70, 70)))
    U, S_, V = O.rpca(A, k=6, l=8, its=1, raw=raw, seed=5)
    exact = O.resid_exact(A, U, S_, V, raw=raw)
    Ac = A if raw else A - A.mean(0)
    assert np.isclose(exact, np.linalg.norm(Ac - (U * S_) @ V.T, 2), rtol=1e-12)
    for iters in (1, 3, 20):
        est = O.resid_power(A, U, S_, V, raw=raw, iters=iters, seed=iters)
        assert est <= exact * (1 + 1e-12)      # |E^T E x| <= ||E||^2 for unit x
        if iters >= 3:                         # within 2x w.h.p.; the failure probability
            assert est >= exact / 2            # falls exponentially with the iteration count
    assert np.isclose(O.resid_power(A, U, S_, V, raw=raw, iters=200, seed=1), exact, rtol=1e-6)


def test_argument_checks():
    A = np.zeros((10, 8))
    with pytest.raises(ValueError):
        O.rpca(A, k=5, l=4)
    with pytest.raises(ValueError):
        O.rpca(A, k=2, l=9)
    with pytest.raises(ValueError):
        O.rpca(A, k=2, l=3, its=-1)

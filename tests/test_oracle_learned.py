"""Pins for the oracle's learned-weighting pieces: finite differences for the MLP
gradient, closed forms for the features, the label on known singular vectors."""
import math

import numpy as np
import pytest

import oracle as O
import synth as S

L = O.learned_oracle


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = L.init_params(1)
    F = rng.standard_normal((40, L.F_IN))
    t = rng.standard_normal(40)
    loss, g = L.loss_grad(p, F, t)
    idx = np.concatenate([rng.choice(L.N_PARAMS, 60, replace=False), [L.N_PARAMS - 1]])
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (L.loss_grad(p + e, F, t)[0] - L.loss_grad(p - e, F, t)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_forward_closed_form_linear_regime():
    # with every pre-activation positive the MLP is the affine map w3^T (W2^T (W1^T f + b1) + b2) + b3
    p = np.abs(L.init_params(2))
    W1, b1, W2, b2, w3, b3 = L.split_params(p)
    f = np.abs(np.random.default_rng(3).standard_normal((5, L.F_IN)))
    y, _ = L.forward(p, f)
    ref = ((f @ W1 + b1) @ W2 + b2) @ w3 + b3
    assert np.allclose(y, ref, rtol=1e-12)


def test_features_closed_forms():
    A = S.kernel_matrix_np(S.KernelSpec(300, 80, 0.3, 5)).astype(np.float64)
    F = L.features(A, raw=False, seed=4)
    # relative energies average to ~0 in log; scaling one column by s shifts its f0 by 2 log s
    B = A.copy()
    B[:, 7] *= 3.0
    G = L.features(B, raw=False, seed=4)
    q = ((A - A.mean(0)) ** 2).sum(0)
    qb = q.copy(); qb[7] *= 9.0
    assert np.isclose(G[7, 0] - F[7, 0], math.log(9.0) - math.log(qb.mean() / q.mean()), atol=1e-9)
    # f1 is the column mean over sqrt(qbar / m); f11, f12 the log sizes
    assert np.allclose(F[:, 1], A.mean(0) / math.sqrt(q.mean() / 300), rtol=1e-9)
    assert np.allclose(F[:, 11], math.log(300) / 8) and np.allclose(F[:, 12], math.log(80) / 8)
    # sketch features have unit mean square per row, and are invariant to scaling A
    assert np.allclose((F[:, 3:11] ** 2).mean(0), 1.0)
    assert np.allclose(L.features(5.0 * A, seed=4)[:, 3:11], F[:, 3:11], rtol=1e-9, atol=1e-12)
    assert np.all(F[:, 13:] == 0)


def test_peak_ratio_feature_closed_forms():
    """f2 = log(m max|a'|^2 / |a'|^2) / 4 of a column: a single spike carries all its
    energy in one entry (log(m) / 4), a column of equal magnitudes none (0), and a
    column with p equal nonzeros gives log(m / p) / 4."""
    m, n = 256, 6
    rng = np.random.default_rng(3)
    A = rng.standard_normal((m, n))
    A[:, 0] = 0.0
    A[17, 0] = -2.5                                   # one spike
    A[:, 1] = np.where(rng.random(m) < 0.5, 1.0, -1.0)   # +-1
    A[:, 2] = 0.0
    A[:32, 2] = 3.0                                   # 32 equal nonzeros
    F = L.features(A, raw=True, seed=2)
    assert np.isclose(F[0, 2], math.log(m) / 4, atol=1e-9)
    assert np.isclose(F[1, 2], 0.0, atol=1e-9)
    assert np.isclose(F[2, 2], math.log(m / 32) / 4, atol=1e-9)
    # centred: a balanced +-1 column has mean 0, so it is unchanged by the centring
    B = A.copy()
    B[:, 1] = np.tile([1.0, -1.0], m // 2)
    assert np.isclose(L.features(B, raw=False, seed=2)[1, 2], 0.0, atol=1e-9)


def test_leverage_target_on_known_vectors():
    n, k = 50, 4
    V = np.zeros((n, k))
    V[np.arange(k), np.arange(k)] = 1.0           # leverage 1 on 4 columns, 0 elsewhere
    t = L.leverage_target(V, k)
    assert np.allclose(t[:k], math.log(n / k + 1e-3)) and np.allclose(t[k:], math.log(1e-3))
    Q, _ = np.linalg.qr(np.random.default_rng(1).standard_normal((n, k)))
    assert np.isclose(np.exp(L.leverage_target(Q, k)).sum(), n + n * 1e-3)


def test_adam_step_decreases_loss():
    rng = np.random.default_rng(7)
    p = L.init_params(3)
    F = rng.standard_normal((200, L.F_IN))
    t = F[:, 0] - 0.5 * F[:, 1]
    m1 = np.zeros_like(p)
    m2 = np.zeros_like(p)
    l0 = L.loss_grad(p, F, t)[0]
    for step in range(1, 201):
        _, g = L.loss_grad(p, F, t)
        p, m1, m2 = L.adam_step(p, g, m1, m2, step, 1e-3)
    assert L.loss_grad(p, F, t)[0] < 0.2 * l0


def test_bf16_round_ties_and_library():
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties to the even mantissa (1)
    assert L.bf16_round(1 + 2.0 ** -8) == 1.0
    # 1 + 3 * 2^-8 is halfway between 1 + 2^-7 (odd) and 1 + 2^-6 (even)
    assert L.bf16_round(1 + 3 * 2.0 ** -8) == 1 + 2.0 ** -6
    assert L.bf16_round(1 + 2.0 ** -8 + 2.0 ** -20) == 1 + 2.0 ** -7
    assert L.bf16_round(-3.0) == -3.0 and L.bf16_round(0.0) == 0.0
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(5).standard_normal(10000).astype(np.float32) * 10.0
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(L.bf16_round(x), ref)


def test_forward_bf16_close_to_exact():
    p = L.init_params(4)
    F = np.random.default_rng(6).standard_normal((300, L.F_IN))
    y, _ = L.forward(p, F)
    yb = L.forward_bf16(p, F)
    # BF16 keeps 8 bits: the outputs agree to a few parts in 1e3 of their scale
    assert np.max(np.abs(y - yb)) < 0.02 * max(1.0, np.max(np.abs(y)))
    assert not np.array_equal(y, yb)


def test_weights_from_output_closed_form_and_clip():
    # d = exp(y) between the clip bounds 1e-2 and 1e2, so the prediction of a
    # leverage label t = log(n lev / k + 1e-3) maps back to n lev / k + 1e-3
    y = np.array([0.0, math.log(5.0), math.log(0.25), 10.0, -10.0, math.log(100.0), math.log(0.01)])
    d = L.weights_from_output(y)
    assert np.allclose(d, [1.0, 5.0, 0.25, 100.0, 0.01, 100.0, 0.01], rtol=1e-12)
    ys = np.linspace(-8, 8, 401)
    ds = L.weights_from_output(ys)
    assert np.all(np.diff(ds) >= 0) and ds.min() == 0.01 and ds.max() == 100.0
    n, k = 50, 4
    Q, _ = np.linalg.qr(np.random.default_rng(3).standard_normal((n, k)))
    lev = (Q ** 2).sum(axis=1)
    assert np.allclose(L.weights_from_output(L.leverage_target(Q, k)),
                       np.clip(n * lev / k + 1e-3, 1e-2, 1e2), rtol=1e-12)


def test_adam_first_step_is_lr_times_sign():
    # with bias correction, m_hat = g and v_hat = g^2 after one step, so every
    # coordinate moves by lr g / (|g| + eps), i.e. lr sign(g) for |g| >> eps
    rng = np.random.default_rng(11)
    p = rng.standard_normal(40)
    g = rng.standard_normal(40) * np.logspace(-3, 3, 40)
    p1, m1, m2 = L.adam_step(p, g, np.zeros(40), np.zeros(40), 1, 1e-3)
    assert np.allclose(p - p1, 1e-3 * np.sign(g), rtol=1e-4, atol=0)
    assert np.allclose(m1, 0.1 * g) and np.allclose(m2, 1e-3 * g * g)

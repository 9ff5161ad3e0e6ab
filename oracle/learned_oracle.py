"""FP64 oracle for the learned column weighting of the sketch (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may use it.

The sketch of Section 2 applies A to i.i.d. Gaussian test vectors; Section 5
notes the algorithms are robust to the law of those vectors.  The learned
variant scales row j of Omega by a weight d_j > 0 (Omega' = diag(d) Omega),
predicted per column of A by a small MLP from cheap column statistics and a
coarse sketch.  This module restates, in plain numpy FP64:

* the per-column features (16 per column, the last three zero):
    c_j    column mean (0 when raw);  a'_ij = a_ij - c_j
    q_j    = sum_i a'_ij^2,  qbar = mean_j q_j,  tau = 1e-12 qbar + 1e-30
    x_j    = max_i |a'_ij|
    S[r,j] = sum_i G[i,r] a'_ij  (G: m x 8 N(0,1) from the Philox stream
             (seed, 2), same mapping as the test matrix)
    rho_r  = sqrt(mean_j S[r,j]^2)
    f0 = log((q_j + tau) / (qbar + tau))
    f1 = c_j / sqrt(qbar / m + tau)
    f2 = log((x_j^2 m + tau) / (q_j + tau)) / 4
    f3..f10 = S[r,j] / (rho_r + 1e-30)
    f11 = log(m) / 8,  f12 = log(n) / 8
* the MLP 16 -> 128 -> 128 -> 1 with ReLU:
    z1 = W1^T f + b1, h1 = relu(z1), z2 = W2^T h1 + b2, h2 = relu(z2),
    y = w3 . h2 + b3;  parameters flattened as [W1 (16x128), b1 (128),
    W2 (128x128), b2 (128), w3 (128), b3 (1)] (row-major)
* the loss mean_j (y_j - t_j)^2 over a batch and its exact gradient
  (hand-derived backpropagation);
* the label: t_j = log(n l_j / k + 1e-3) with l_j = |V_k[j, :]|^2 the
  leverage of column j in the top-k right singular subspace;
* the weight: d_j = clip(exp(y_j), 1e-2, 1e2);
* forward_bf16: the same forward with the inference kernel's rounding points
  (features, W1, W2 and h1 rounded to BF16 by round-to-nearest-even of the
  FP32 value, biases and w3 in FP32), everything else in FP64.
"""
from __future__ import annotations

import math

import numpy as np

from .rpca_oracle import gaussian_omega

F_IN = 16
H = 128
N_PARAMS = F_IN * H + H + H * H + H + H + 1
SKETCH_ROWS = 8


def split_params(p: np.ndarray):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + F_IN * H].reshape(F_IN, H); o += F_IN * H
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    w3 = p[o:o + H]; o += H
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def init_params(seed: int = 0) -> np.ndarray:
    """He-style initialisation (scale sqrt(2 / fan_in)), zero biases."""
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((F_IN, H)) * math.sqrt(2.0 / F_IN)
    W2 = rng.standard_normal((H, H)) * math.sqrt(2.0 / H)
    w3 = rng.standard_normal(H) * math.sqrt(1.0 / H)
    return np.concatenate([W1.ravel(), np.zeros(H), W2.ravel(), np.zeros(H), w3, [0.0]])


def features(A, raw: bool = False, seed: int = 0) -> np.ndarray:
    """n x 16 feature matrix of the columns of A (see the module docstring)."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    c = np.zeros(n) if raw else A.mean(axis=0)
    Ac = A - c[None, :]
    q = (Ac * Ac).sum(axis=0)
    qbar = q.mean()
    tau = 1e-12 * qbar + 1e-30
    x = np.abs(Ac).max(axis=0)
    G = gaussian_omega(m, SKETCH_ROWS, seed, stream=2)
    S = G.T @ Ac                                   # 8 x n
    rho = np.sqrt((S * S).mean(axis=1))
    F = np.zeros((n, F_IN))
    F[:, 0] = np.log((q + tau) / (qbar + tau))
    F[:, 1] = c / math.sqrt(qbar / m + tau)
    F[:, 2] = np.log((x * x * m + tau) / (q + tau)) / 4.0
    F[:, 3:3 + SKETCH_ROWS] = (S / (rho[:, None] + 1e-30)).T
    F[:, 11] = math.log(m) / 8.0
    F[:, 12] = math.log(n) / 8.0
    return F


def forward(p: np.ndarray, F: np.ndarray):
    """MLP output y (N) and the intermediates (z1, h1, z2, h2)."""
    W1, b1, W2, b2, w3, b3 = split_params(p)
    z1 = F @ W1 + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2 + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ w3 + b3
    return y, (z1, h1, z2, h2)


def loss_grad(p: np.ndarray, F: np.ndarray, t: np.ndarray):
    """(mean squared error, gradient w.r.t. the flattened parameters)."""
    W1, b1, W2, b2, w3, b3 = split_params(p)
    F = np.asarray(F, dtype=np.float64)
    y, (z1, h1, z2, h2) = forward(p, F)
    N = F.shape[0]
    r = y - np.asarray(t, dtype=np.float64)
    loss = float((r * r).mean())
    dy = 2.0 * r / N                               # dL/dy
    dw3 = h2.T @ dy
    db3 = dy.sum()
    dz2 = np.outer(dy, w3) * (z2 > 0)
    dW2 = h1.T @ dz2
    db2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2.T) * (z1 > 0)
    dW1 = F.T @ dz1
    db1 = dz1.sum(axis=0)
    g = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dw3, [db3]])
    return loss, g


def bf16_round(x) -> np.ndarray:
    """Round to BF16 (8 significant bits) by round-to-nearest-even of the FP32 value;
    returned as FP64.  Finite inputs only."""
    x32 = np.asarray(x, dtype=np.float32)
    bits = x32.view(np.uint32).astype(np.uint64)
    lsb = (bits >> 16) & 1
    r = ((bits + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def forward_bf16(p: np.ndarray, F: np.ndarray) -> np.ndarray:
    """MLP output with the tensor-core kernel's rounding points (module docstring)."""
    W1, b1, W2, b2, w3, b3 = split_params(p)
    f32 = lambda v: np.asarray(v, dtype=np.float32).astype(np.float64)   # noqa: E731
    z1 = bf16_round(F) @ bf16_round(W1) + f32(b1)
    h1 = bf16_round(np.maximum(f32(z1), 0.0))
    z2 = h1 @ bf16_round(W2) + f32(b2)
    return np.maximum(z2, 0.0) @ f32(w3) + f32(b3)


def leverage_target(V: np.ndarray, k: int) -> np.ndarray:
    """t_j = log(n |V_k[j, :]|^2 / k + 1e-3) from the top-k right singular vectors."""
    V = np.asarray(V, dtype=np.float64)[:, :k]
    n = V.shape[0]
    return np.log(n * (V * V).sum(axis=1) / k + 1e-3)


def weights_from_output(y: np.ndarray) -> np.ndarray:
    return np.clip(np.exp(np.asarray(y, dtype=np.float64)), 1e-2, 1e2)


def adam_step(p, g, m1, m2, step: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam update (Kingma & Ba 2015) with bias correction; returns (p, m1, m2)."""
    m1 = b1 * m1 + (1 - b1) * g
    m2 = b2 * m2 + (1 - b2) * g * g
    mh = m1 / (1 - b1 ** step)
    vh = m2 / (1 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m1, m2

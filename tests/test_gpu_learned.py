"""Parity of the learned sketch weighting's kernels with the oracle.

Features (dense and batched), the tensor-core MLP forward (against the oracle's
forward with the same BF16 rounding points), the training gradient and Adam
step, the leverage labels, and the learned PCA with its fallback: the
weighted sketch's output against the oracle on the same weights, and the
fallback firing on a network built to weight the wrong columns.
"""
import numpy as np
import pytest

import oracle as O
import synth as S
from gpu_util import cuda, subspace_dist, subspace_tol, to_dev, to_np

pytestmark = pytest.mark.gpu
LO = O.learned_oracle


def _feat_close(Fg, Fo):
    err = np.abs(Fg - Fo) / np.maximum(1.0, np.abs(Fo))
    assert err.max() < 2e-4, (err.max(), np.unravel_index(err.argmax(), err.shape))


@pytest.mark.parametrize("shape,raw", [((700, 300), False), ((700, 300), True), ((5000, 1000), False),
                                       ((257, 129), False), ((64, 5), True)])
def test_dense_features_match_oracle(shape, raw):
    cuda()
    import paper_1412_3510_gb300 as rp
    m, n = shape
    A = S.kernel_matrix_np(S.KernelSpec(m, n, 0.2, 17 + m))
    A[:, 3] = 0.75                                   # a constant column (q = 0 when centred)
    Fg = to_np(rp.rpca_sketch_features(to_dev(A), raw=raw, seed=21))
    Fo = LO.features(A, raw=raw, seed=21)
    _feat_close(Fg, Fo)


def test_dense_features_strided_and_unaligned():
    torch = cuda()
    import paper_1412_3510_gb300 as rp
    A = S.kernel_matrix_np(S.KernelSpec(400, 203, 0.3, 5))
    big = torch.zeros(400, 211, device="cuda")
    big[:, 1:204] = to_dev(A)
    view = big[:, 1:204]                             # lda 211, base not 16-byte aligned
    Fg = to_np(rp.rpca_sketch_features(view, seed=3))
    _feat_close(Fg, LO.features(A, seed=3))


def test_batched_features_match_oracle():
    cuda()
    import paper_1412_3510_gb300 as rp
    specs = [S.KernelSpec(300, 1100, 0.3, 1), S.KernelSpec(40, 7, 0.1, 2), S.KernelSpec(1000, 64, 0.5, 3),
             S.KernelSpec(129, 300, 0.05, 4)]
    mats = [S.kernel_matrix_np(sp) for sp in specs]
    batch = rp.Batch([to_dev(a) for a in mats], 4)
    for raw in (False, True):
        F = to_np(rp.rpca_batched_features(batch, raw=raw, seed=8))
        o = 0
        for a in mats:
            n = a.shape[1]
            _feat_close(F[o:o + n], LO.features(a, raw=raw, seed=8))
            o += n


@pytest.mark.parametrize("N", [1, 1000, 128 * 400 + 7])
def test_mlp_forward_matches_oracle(N):
    torch = cuda()
    import paper_1412_3510_gb300 as rp
    p = LO.init_params(11)
    p[LO.F_IN * LO.H:LO.F_IN * LO.H + LO.H] = 0.1    # nonzero biases exercise the epilogues
    p[-1] = 0.3
    F = np.random.default_rng(N).standard_normal((N, LO.F_IN)).astype(np.float32)
    F[:, 13:] = 0.0
    pt = to_dev(p.astype(np.float32))
    packed = rp.rpca_mlp_pack(pt)
    y, d = rp.rpca_mlp_forward(packed, to_dev(F))
    yo = LO.forward_bf16(p.astype(np.float32).astype(np.float64), F.astype(np.float64))
    yg = to_np(y)
    err = np.abs(yg - yo)
    assert err.max() < 1e-3 * max(1.0, np.abs(yo).max()), err.max()
    assert np.allclose(to_np(d), LO.weights_from_output(yg), rtol=1e-5)


def test_mlp_loss_grad_matches_oracle():
    torch = cuda()
    import paper_1412_3510_gb300 as rp
    rng = np.random.default_rng(2)
    for N in (37, 64 * 5 + 9):
        p = (LO.init_params(3) + 0.01 * rng.standard_normal(LO.N_PARAMS)).astype(np.float32)
        F = rng.standard_normal((N, LO.F_IN)).astype(np.float32)
        t = rng.standard_normal(N).astype(np.float32)
        loss, g = rp.rpca_mlp_loss_grad(to_dev(p), to_dev(F), to_dev(t))
        lo, go = LO.loss_grad(p.astype(np.float64), F.astype(np.float64), t.astype(np.float64))
        gg = to_np(g)
        assert abs(float(loss.item()) - lo) <= 1e-5 * lo
        assert np.linalg.norm(gg - go) <= 1e-4 * np.linalg.norm(go)
        assert np.max(np.abs(gg - go)) <= 1e-4 * np.max(np.abs(go))
        _, g2 = rp.rpca_mlp_loss_grad(to_dev(p), to_dev(F), to_dev(t))
        assert torch.equal(g, g2)                    # fixed-order reduction


def test_mlp_adam_matches_oracle():
    torch = cuda()
    import paper_1412_3510_gb300 as rp
    rng = np.random.default_rng(4)
    p = LO.init_params(5)
    F = rng.standard_normal((200, LO.F_IN)).astype(np.float32)
    t = (F[:, 0] - F[:, 1]).astype(np.float32)
    pg = to_dev(p.astype(np.float32))
    m1 = torch.zeros_like(pg)
    m2 = torch.zeros_like(pg)
    po, m1o, m2o = p.astype(np.float32).astype(np.float64), np.zeros(LO.N_PARAMS), np.zeros(LO.N_PARAMS)
    for step in range(1, 6):
        _, g = rp.rpca_mlp_loss_grad(pg, to_dev(F), to_dev(t))
        gn = to_np(g)
        rp.rpca_mlp_adam(pg, g, m1, m2, step, 1e-3)
        po, m1o, m2o = LO.adam_step(po, gn, m1o, m2o, step, 1e-3)
        assert np.max(np.abs(to_np(pg) - po)) < 1e-6, step
    l0 = LO.loss_grad(p, F, t)[0]
    assert LO.loss_grad(to_np(pg), F, t)[0] < l0


def test_leverage_target_matches_oracle():
    cuda()
    import paper_1412_3510_gb300 as rp
    Q, _ = np.linalg.qr(np.random.default_rng(1).standard_normal((300, 9)))
    V = np.zeros((300, 12), dtype=np.float32)
    V[:, :9] = Q
    tg = to_np(rp.rpca_leverage_target(to_dev(V), 7))
    assert np.allclose(tg, LO.leverage_target(V.astype(np.float64), 7), rtol=1e-5, atol=1e-5)


def _packed(rp, p):
    return rp.rpca_mlp_pack(to_dev(np.asarray(p, dtype=np.float32)))


def test_dense_learned_matches_weighted_oracle():
    torch = cuda()
    import paper_1412_3510_gb300 as rp
    A = S.kernel_matrix_np(S.KernelSpec(900, 350, 0.2, 31))
    k, l, its, seed = 10, 14, 1, 6
    p = LO.init_params(7)
    p[-1] = -0.5
    packed = _packed(rp, p)
    Ad = to_dev(A)
    U, Sg, V, info = rp.rpca_dense_learned(Ad, packed, k, l, its=its, seed=seed, resid_iters=10,
                                           fallback_ratio=1e6)
    assert not info["fell_back"]
    # the weights the call used, from the same kernels
    _, d = rp.rpca_mlp_forward(packed, rp.rpca_sketch_features(Ad, seed=seed))
    U2, S2, V2 = rp.rpca_dense(Ad, k, l, its=its, seed=seed, col_weights=d)
    assert torch.equal(U, U2) and torch.equal(Sg, S2) and torch.equal(V, V2)
    # the oracle on the same weighted test matrix
    om = O.gaussian_omega(350, l, seed) * to_np(d)[:, None]
    Uo, so, Vo = O.rpca(A, k, l, its, omega=om)
    sg = to_np(Sg)
    assert np.all(np.abs(sg - so) <= 1e-4 * so + 1e-6 * so[0])
    kk, tol = subspace_tol(so, k)
    if kk:
        assert subspace_dist(to_np(V)[:, :kk], Vo[:, :kk]) < tol
    # the estimate is the Section 4 estimator of the returned factors
    est = rp.rpca_resid_norm(Ad, U, Sg, V, iters=10, seed=seed)
    assert abs(est - info["est"]) <= 1e-6 * est
    assert info["s_k1"] > 0


def test_dense_learned_fallback_fires():
    torch = cuda()
    import paper_1412_3510_gb300 as rp
    # the top-k subspace lives in 12 high-energy columns; a network that gives
    # high-energy columns (feature 0 > 0) the weight 1e-2 hides it from the sketch
    rng = np.random.default_rng(12)
    m, n, k, l = 600, 300, 5, 7
    A = rng.standard_normal((m, n))                 # noise: singular values <= ~42
    loud = rng.choice(n, 12, replace=False)
    A[:, loud] += rng.standard_normal((m, 5)) @ rng.standard_normal((5, 12)) * 2.0   # signal: 94..267
    A = A.astype(np.float32)
    p = np.zeros(LO.N_PARAMS)
    W1, b1, W2, b2, w3, b3 = LO.split_params(p)      # views into p
    W1[0, 0] = 1.0                                   # h1_0 = relu(f0)
    W2[0, 0] = 1.0
    w3[0] = -10.0                                    # y = -10 relu(f0): d = 1e-2 on loud columns
    Fo = LO.features(A, seed=2)
    assert np.all(Fo[loud, 0] > 0.5) and np.all(np.delete(Fo[:, 0], loud) < 0.3)
    Ad = to_dev(A)
    for its in (0, 1):
        U, Sg, V, info = rp.rpca_dense_learned(Ad, _packed(rp, p), k, l, its=its, seed=2, resid_iters=12)
        assert info["fell_back"], info
        U2, S2, V2 = rp.rpca_dense(Ad, k, l, its=its, seed=2)
        assert torch.equal(U, U2) and torch.equal(Sg, S2) and torch.equal(V, V2)
    # a network that outputs 0 gives d = 1 (the plain sketch): no fallback on a
    # matrix with a decaying spectrum, and the plain output
    B = to_dev(S.kernel_matrix_np(S.KernelSpec(600, 300, 0.5, 9)))
    U, Sg, V, info = rp.rpca_dense_learned(B, _packed(rp, np.zeros(LO.N_PARAMS)), k, k + 6, its=2, seed=2,
                                           resid_iters=12)
    assert not info["fell_back"], info
    U2, S2, V2 = rp.rpca_dense(B, k, k + 6, its=2, seed=2)
    assert torch.equal(U, U2) and torch.equal(Sg, S2) and torch.equal(V, V2)


def test_batched_learned_fallback_fires_per_matrix():
    """The batched form's fallback: matrices whose learned weights hide the signal (weight
    1e-2 on the 12 columns that carry the top-k subspace) are recomputed with the plain
    sketch and flagged; matrices with neutral weights keep their result.  Both end equal,
    bit for bit, to plain rpca_batched."""
    torch = cuda()
    import paper_1412_3510_gb300 as rp
    k, l, its = 5, 11, 1
    mats, weights, bad = [], [], []
    for i in range(4):                                   # signal hidden by the weights
        rng = np.random.default_rng(40 + i)
        m, n = 500 + 37 * i, 300 - 11 * i
        A = rng.standard_normal((m, n))
        loud = rng.choice(n, 12, replace=False)
        A[:, loud] += rng.standard_normal((m, 5)) @ rng.standard_normal((5, 12)) * 2.0
        d = np.ones(n, dtype=np.float32)
        d[loud] = 1e-2
        mats.append(A.astype(np.float32))
        weights.append(d)
        bad.append(True)
    for i in range(4):                                   # neutral weights, decaying spectra
        A = S.kernel_matrix_np(S.KernelSpec(400 + 50 * i, 200 + 20 * i, 0.3 + 0.1 * i, 60 + i))
        mats.append(A)
        weights.append(np.ones(A.shape[1], dtype=np.float32))
        bad.append(False)
    dev = [to_dev(a) for a in mats]
    wdev = [to_dev(d) for d in weights]
    b1 = rp.Batch(dev, k)
    U1, S1, V1, est = rp.rpca_batched_learned(b1, wdev, l, its=its, seed=3, resid_iters=3, fallback_ratio=1.1)
    st = b1.status.cpu().numpy()
    e = est.cpu().numpy()
    assert np.array_equal(st, np.where(bad, 1, 0)), (st, e)
    assert np.all(e[:4, 0] > 1.1 * e[:4, 1]) and np.all(e[4:, 0] <= 1.1 * e[4:, 1])
    b2 = rp.Batch(dev, k)
    U2, S2, V2 = rp.rpca_batched(b2, l, its=its, seed=3)
    for i in range(len(mats)):
        assert torch.equal(U1[i], U2[i]) and torch.equal(S1[i], S2[i]) and torch.equal(V1[i], V2[i]), i
    # the estimate is Section 4's estimator: it never exceeds the residual's norm
    for i in range(4, 8):
        Ai = mats[i].astype(np.float64)
        Ac = Ai - Ai.mean(0)
        E = Ac - (to_np(U1[i]) * to_np(S1[i])) @ to_np(V1[i]).T
        assert e[i, 0] <= np.linalg.norm(E, 2) * (1 + 1e-4)


def test_dense_learned_rejects_bad_args():
    cuda()
    import paper_1412_3510_gb300 as rp
    A = to_dev(S.kernel_matrix_np(S.KernelSpec(100, 50, 0.3, 1)))
    packed = _packed(rp, LO.init_params(0))
    with pytest.raises(rp.RpcaError):
        rp.rpca_dense_learned(A, packed, 5, 7, resid_iters=0)
    with pytest.raises(rp.RpcaError):
        rp.rpca_dense_learned(A, packed, 5, 7, fallback_ratio=0.0)
    with pytest.raises(rp.RpcaError):
        rp.rpca_dense_learned(A, packed[1:], 5, 7)   # misaligned blob


def test_training_reduces_loss_and_beats_plain_at_equal_its():
    """Train on a family, then compare learned and plain sketches on held-out matrices."""
    torch = cuda()
    import paper_1412_3510_gb300 as rp
    from paper_1412_3510_gb300 import learned as LR
    k, l = 8, 10
    tr = [to_dev(S.kernel_matrix_np(sp)) for sp in S.kernel_batch_specs(150, 41, (256, 800), (64, 300))]
    params, packed, info = LR.train_sketch_mlp(tr, k, steps=1500, batch=2048, lr=1e-3, seed=3)
    F, t = LR.leverage_dataset(tr[:20], k, seed=3)
    l_end = float(rp.rpca_mlp_loss_grad(params, F, t)[0].item())
    assert l_end < 0.8 * info["target_var"], (l_end, info["target_var"])
    # held-out: residual / s_{k+1} (exact, FP64) for plain and learned at its = 1
    te_specs = S.kernel_batch_specs(32, 42, (256, 800), (64, 300))
    te = [S.kernel_matrix_np(sp) for sp in te_specs]
    batch = rp.Batch([to_dev(a) for a in te], k)
    d, _ = LR.batched_learned_weights(batch, packed, seed=5)
    ratios = {}
    for name, w in (("plain", None), ("learned", d)):
        U, Sg, V = rp.rpca_batched(batch, l, its=1, seed=5, col_weights=w)
        r = []
        for a, u, s, v in zip(te, U, Sg, V):
            ac = a.astype(np.float64) - a.mean(0)
            sk1 = np.linalg.svd(ac, compute_uv=False)[k]
            r.append(np.linalg.norm(ac - (to_np(u) * to_np(s)) @ to_np(v).T, 2) / sk1)
        ratios[name] = np.array(r)
    assert np.all(batch.status.cpu().numpy() == 0)
    # the learned weighting must not be worse on the tail of the distribution
    assert np.quantile(ratios["learned"], 0.9) <= np.quantile(ratios["plain"], 0.9) * 1.02, ratios

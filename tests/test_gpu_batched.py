"""Parity of the batched path (rpca_batched: one persistent launch) with the oracle.

Every matrix of a batch of uneven Gaussian-kernel matrices (the batched
workload's family) is checked against the FP64 oracle on the same matrix and
seed, with the dense path's bars; a malformed descriptor is skipped and
reported without disturbing the others.
"""
import numpy as np
import pytest

import oracle as O
import synth as S
from gpu_util import cuda, subspace_dist, subspace_tol, to_dev, to_np

pytestmark = pytest.mark.gpu


def _batch(count, seed, m_range=(40, 700), n_range=(30, 300)):
    specs = S.kernel_batch_specs(count, seed, m_range=m_range, n_range=n_range)
    return [S.kernel_matrix_np(sp) for sp in specs]


@pytest.mark.parametrize("its", [0, 1, 2])
def test_batched_matches_oracle(its):
    cuda()
    import paper_1412_3510_gb300 as rp
    k, l = 6, 8
    mats = _batch(24, 100 + its)
    batch = rp.Batch([to_dev(a) for a in mats], k)
    U, Sg, V = rp.rpca_batched(batch, l, its=its, seed=9)
    st = batch.status.cpu().numpy()
    assert np.all(st == 0)
    for a, u, s, v in zip(mats, U, Sg, V):
        Uo, so, Vo = O.rpca(a, k, l, its, raw=False, seed=9)
        sg = to_np(s)
        assert np.all(np.abs(sg - so) <= 1e-4 * so + 1e-6 * so[0]), (np.abs(sg - so) / so).max()
        ug, vg = to_np(u), to_np(v)
        assert np.linalg.norm(ug.T @ ug - np.eye(k), 2) < 1e-4
        kk, tol = subspace_tol(so, k)
        if kk:
            assert subspace_dist(ug[:, :kk], Uo[:, :kk]) < tol
            assert subspace_dist(vg[:, :kk], Vo[:, :kk]) < tol
        idx = np.argmax(np.abs(vg), axis=0)
        assert np.all(vg[idx, np.arange(k)] > 0)


def test_batched_agrees_with_single_matrix_path_and_widths():
    cuda()
    import paper_1412_3510_gb300 as rp
    mats = _batch(10, 7, m_range=(100, 3000), n_range=(64, 1024))
    for k, l in ((1, 1), (16, 20), (30, 32)):
        lp = (l + 1 + 7) // 8 * 8
        ok = [a for a in mats if min(a.shape) >= l and a.shape[1] * lp <= 24576]
        batch = rp.Batch([to_dev(a) for a in ok], k)
        _, Sb, _ = rp.rpca_batched(batch, l, its=2, seed=3)
        for a, s in zip(ok, Sb):
            _, s1, _ = rp.rpca_dense(to_dev(a), k, l, its=2, seed=3)
            assert np.allclose(to_np(s), to_np(s1), rtol=2e-5, atol=1e-6 * float(s1[0]))


def test_batched_skips_bad_descriptor():
    cuda()
    import paper_1412_3510_gb300 as rp
    mats = _batch(5, 2)
    mats[2] = mats[2][:5, :5]                  # l = 8 > min(m, n): invalid for this item
    batch = rp.Batch([to_dev(a) for a in mats], 4)
    with pytest.raises(rp.RpcaError):
        rp.rpca_batched(batch, 8, its=1, seed=1)
    st = batch.status.cpu().numpy()
    assert st[2] == -1 and np.all(np.delete(st, 2) == 0)
    _, so, _ = O.rpca(mats[0], 4, 8, 1, seed=1)
    assert np.allclose(to_np(batch.S[0]), so, rtol=1e-4)


def test_batched_column_weights():
    cuda()
    import paper_1412_3510_gb300 as rp
    mats = _batch(6, 4)
    ws_ = [np.linspace(0.5, 2.0, a.shape[1]).astype(np.float32) for a in mats]
    batch = rp.Batch([to_dev(a) for a in mats], 5)
    _, Sg, _ = rp.rpca_batched(batch, 7, its=1, seed=2, col_weights=[to_dev(w) for w in ws_])
    for a, w, s in zip(mats, ws_, Sg):
        om = O.gaussian_omega(a.shape[1], 7, 2) * w[:, None].astype(np.float64)
        _, so, _ = O.rpca(a, 5, 7, 1, omega=om)
        assert np.allclose(to_np(s), so, rtol=1e-4, atol=1e-6 * so[0])


def test_batched_tuner_keeps_results_identical():
    """The autotuner times the tile shapes on the batch; every shape gives bit-identical
    outputs (each output sums in the same order), and later calls use the choice."""
    torch = cuda()
    import paper_1412_3510_gb300 as rp
    mats = _batch(40, 7, m_range=(100, 3000), n_range=(30, 600))
    batch = rp.Batch([to_dev(a) for a in mats], 6)
    U1, S1, V1 = rp.rpca_batched(batch, 8, its=1, seed=3)
    ref = [(u.clone(), s.clone(), v.clone()) for u, s, v in zip(U1, S1, V1)]
    shape, ms = rp.rpca_batched_tune(batch, 8, its=1, seed=3)
    assert shape in ((2, 64), (4, 32), (8, 32)) and len(ms) == 3 and all(t > 0 for t in ms)
    for (u, s, v), (u0, s0, v0) in zip(zip(batch.U, batch.S, batch.V), ref):    # last tuning run: 8 x 32
        assert torch.equal(u, u0) and torch.equal(s, s0) and torch.equal(v, v0)
    U3, S3, V3 = rp.rpca_batched(batch, 8, its=1, seed=3)                      # the tuned shape
    for (u, s, v), (u0, s0, v0) in zip(zip(U3, S3, V3), ref):
        assert torch.equal(u, u0) and torch.equal(s, s0) and torch.equal(v, v0)
    assert np.all(batch.status.cpu().numpy() == 0)

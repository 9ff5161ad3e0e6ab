"""Parity of the CUDA sparse path (rpca_csr, rpca_resid_norm_csr) with the oracle on CSR input.

The oracle keeps A as a scipy CSR matrix (Section 5: the same code serves
dense and sparse A); both sides see the same FP32 values and Philox seed.
Bars as for the dense FP32 path: sigma within 1e-4 relative (+1e-6 ||A||),
subspaces within 1e-3, residual estimate within 1e-3 relative.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
import synth as S
from gpu_util import cuda, subspace_dist, subspace_tol, to_np

pytestmark = pytest.mark.gpu


def _dev(csr):
    import torch
    return (torch.from_numpy(csr.indptr.astype(np.int32)).cuda(), torch.from_numpy(csr.indices.astype(np.int32)).cuda(),
            torch.from_numpy(csr.data.astype(np.float32)).cuda())


def _check(csr, k, l, its, raw, seed, **kw):
    cuda()
    import paper_1412_3510_gb300 as rp
    rp_, ci, va = _dev(csr)
    U, Sg, V = rp.rpca_csr(rp_, ci, va, csr.shape, k, l, its=its, raw=raw, seed=seed, **kw)
    Ug, sg, Vg = to_np(U), to_np(Sg), to_np(V)
    Uo, so, Vo = O.rpca(csr, k, l, its, raw=raw, seed=seed)
    assert np.all(np.abs(sg - so) <= 1e-4 * so + 1e-6 * so[0]), (np.abs(sg - so) / so).max()
    assert np.linalg.norm(Ug.T @ Ug - np.eye(k), 2) < 1e-4
    kk, tol = subspace_tol(so, k)
    if kk:
        assert subspace_dist(Ug[:, :kk], Uo[:, :kk]) < tol
        assert subspace_dist(Vg[:, :kk], Vo[:, :kk]) < tol
    # sign rule: the largest-magnitude entry of every right vector is positive
    piv = np.abs(Vg).argmax(axis=0)
    assert np.all(Vg[piv, np.arange(k)] > 0)
    est = rp.rpca_resid_norm_csr(rp_, ci, va, csr.shape, U, Sg, V, raw=raw, iters=20, seed=3)
    ref = O.resid_power(csr, Ug.astype(np.float32), sg.astype(np.float32), Vg.astype(np.float32), raw=raw,
                        iters=20, seed=3)
    assert abs(est - ref) <= 1e-3 * ref


@pytest.mark.parametrize("renorm", ["cholqr", "lu"])
@pytest.mark.parametrize("raw", [True, False])
def test_powerlaw_csr_parity(raw, renorm):
    rp_, ci, va = S.powerlaw_csr(3000, 1500, 40000, exponent=2.1, rank=8, seed=5)
    csr = sp.csr_matrix((va, ci, rp_), shape=(3000, 1500))
    _check(csr, 8, 10, 3, raw, seed=11, renorm=renorm)


def test_tall_csr_parity():
    """60000 rows: the m-side renormalisations run on the tensor cores."""
    rp_, ci, va = S.powerlaw_csr(60000, 2000, 300000, exponent=2.1, rank=6, seed=8)
    csr = sp.csr_matrix((va, ci, rp_), shape=(60000, 2000))
    _check(csr, 6, 10, 2, False, seed=3)


def test_tall_powerlaw_csr_parity():
    """400000 rows, l = 30: heavy rows of A^T (power-law columns) much longer than a chunk,
    and the m-side block (51 MB) on the tensor-core renormalisations."""
    rp_, ci, va = S.powerlaw_csr(400000, 3000, 2000000, exponent=2.1, rank=8, seed=21)
    csr = sp.csr_matrix((va, ci, rp_), shape=(400000, 3000))
    assert np.diff(csr.tocsc().indptr).max() > 256       # heavy rows of A^T exist
    _check(csr, 10, 30, 2, False, seed=5)


def test_wide_csr_parity():
    """n = 60000 columns: the sign rule scans right vectors longer than one pass of its
    1024-thread CTA (eight strided loads per thread per step)."""
    rp_, ci, va = S.powerlaw_csr(20000, 60000, 400000, exponent=2.1, rank=6, seed=17)
    csr = sp.csr_matrix((va, ci, rp_), shape=(20000, 60000))
    _check(csr, 6, 10, 2, True, seed=9)


def test_heavy_rows_and_empty_rows():
    # rows with many more than 2048 nonzeros (split into chunks), empty rows, a column of A^T > 2048
    rng = np.random.default_rng(9)
    m, n = 1200, 5000
    rows, cols = [], []
    for r in (3, 700):                           # two heavy rows
        c = rng.choice(n, size=4500, replace=False)
        rows += [r] * c.size
        cols += list(c)
    for r in range(0, m, 2):                    # light rows; odd rows stay empty
        c = rng.choice(n, size=rng.integers(1, 12), replace=False)
        rows += [r] * c.size
        cols += list(c)
    rows += list(range(0, m, 3))                 # a heavy column of A (heavy row of A^T)
    cols += [17] * len(range(0, m, 3))
    vals = rng.standard_normal(len(rows)).astype(np.float32)
    csr = sp.csr_matrix((vals, (rows, cols)), shape=(m, n))
    csr.sum_duplicates()
    _check(csr, 6, 8, 2, False, seed=2)


def test_duplicates_and_unsorted_columns_are_summed():
    cuda()
    import torch
    import paper_1412_3510_gb300 as rp
    rng = np.random.default_rng(1)
    dense = rng.standard_normal((200, 90)).astype(np.float32) * (rng.random((200, 90)) < 0.2)
    csr = sp.csr_matrix(dense)
    # split every value into two duplicate entries, shuffle column order within rows
    ip, ix, dv = [0], [], []
    for r in range(csr.shape[0]):
        a, b = csr.indptr[r], csr.indptr[r + 1]
        cols = np.concatenate([csr.indices[a:b], csr.indices[a:b]])
        vals = np.concatenate([0.25 * csr.data[a:b], 0.75 * csr.data[a:b]]).astype(np.float32)
        perm = rng.permutation(cols.size)
        ix += list(cols[perm]); dv += list(vals[perm]); ip.append(len(ix))
    t = lambda a, d: torch.tensor(np.asarray(a), dtype=d, device="cuda")
    _, s1, _ = rp.rpca_csr(t(ip, torch.int32), t(ix, torch.int32), t(dv, torch.float32), (200, 90), 5, 7, seed=4)
    _, s2, _ = rp.rpca_csr(*[x for x in _dev(csr)], (200, 90), 5, 7, seed=4)
    assert torch.allclose(s1, s2, rtol=2e-6)


def test_invalid_column_index_is_reported_not_read():
    cuda()
    import torch
    import paper_1412_3510_gb300 as rp
    ip = torch.tensor([0, 2, 3, 5], dtype=torch.int32, device="cuda")
    ix = torch.tensor([0, 9, 1, 2, 3], dtype=torch.int32, device="cuda")     # 9 >= n = 4
    va = torch.ones(5, device="cuda")
    with pytest.raises(rp.RpcaError) as e:
        rp.rpca_csr(ip, ix, va, (3, 4), 1, 2)
    assert e.value.code == -1


def test_csr_agrees_with_dense_path():
    cuda()
    import torch
    import paper_1412_3510_gb300 as rp
    rp_, ci, va = S.powerlaw_csr(800, 600, 9000, rank=5, seed=3)
    csr = sp.csr_matrix((va, ci, rp_), shape=(800, 600))
    U1, S1, V1 = rp.rpca_csr(*_dev(csr), (800, 600), 5, 8, its=2, seed=7)
    U2, S2, V2 = rp.rpca_dense(torch.from_numpy(csr.toarray()).cuda(), 5, 8, its=2, seed=7)
    assert torch.allclose(S1, S2, rtol=1e-5)

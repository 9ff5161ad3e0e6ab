"""Parity of the CUDA residual estimator (Section 4 power method) with the oracle's."""
import numpy as np
import pytest

import oracle as O
import synth as S
from gpu_util import cuda, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m,n,k,raw,iters", [(300, 200, 6, False, 20), (257, 333, 5, True, 7),
                                             (1000, 400, 20, False, 30), (64, 64, 1, True, 3)])
def test_estimator_matches_oracle_on_same_factors(m, n, k, raw, iters):
    cuda()
    import paper_1412_3510_gb300 as rp
    sig = np.exp(-np.arange(1, min(m, n) + 1) / 10.0)
    A = S.haar_dense_np(m, n, sig, seed=m + n)
    if not raw:
        A = A + np.float32(0.5)
    U, s, V = O.rpca(A, k, k + 2, 1, raw=raw, seed=3)
    U32, s32, V32 = (x.astype(np.float32) for x in (U, s, V))
    est = rp.rpca_resid_norm(to_dev(A), to_dev(U32), to_dev(s32), to_dev(V32), raw=raw, iters=iters, seed=9)
    ref = O.resid_power(A, U32, s32, V32, raw=raw, iters=iters, seed=9)
    assert abs(est - ref) <= 1e-3 * ref
    exact = O.resid_exact(A, U32, s32, V32, raw=raw)
    assert est <= exact * (1 + 1e-4)


def test_estimator_k0_is_norm_of_centred_matrix():
    cuda()
    import torch
    import paper_1412_3510_gb300 as rp
    A = np.random.default_rng(2).standard_normal((120, 80)).astype(np.float32) + 1.0
    e = torch.empty(0, device="cuda")
    est = rp.rpca_resid_norm(to_dev(A), e.view(120, 0), e, e.view(80, 0), raw=False, iters=200, seed=1)
    assert abs(est - np.linalg.norm(A - A.mean(0), 2)) < 1e-4 * est


def test_pipeline_residual_matches_oracle():
    cuda()
    import paper_1412_3510_gb300 as rp
    w = S.WORKLOADS["dense_2000x1000_k10"]
    A = S.haar_dense_np(w["m"], w["n"], w["spectrum"](1000), w["seed"])
    Ad = to_dev(A)
    U, Sg, V = rp.rpca_dense(Ad, w["k"], w["l"], its=w["its"], seed=1)
    est = rp.rpca_resid_norm(Ad, U, Sg, V, raw=False, iters=20, seed=2)
    Uo, so, Vo = O.rpca(A, w["k"], w["l"], w["its"], seed=1)
    ref = O.resid_power(A, Uo, so, Vo, raw=False, iters=20, seed=2)
    assert abs(est - ref) <= 1e-3 * ref
    sk1 = O.exact_singular_values(A)[w["k"]]
    assert est <= 1.1 * sk1

"""The split-BF16 form at full size: 200000 x 20000 (A = 16 GB FP32), k = 200, l = 210,
its = 2, centred, in the launch configuration the benchmark times.

The FP64 oracle cannot run at this size, so the outputs are checked through
properties that hold at any size, on samples where a property needs the data:
 - U and V have orthonormal columns and S is descending;
 - A_c^T U = V diag(S) holds exactly for this method (B = Q^* A_c and
   B^* = Q2 Z Sigma W^*, so A_c^* Q W = Q2 Z Sigma), checked on sampled columns
   of A recomputed in FP64 on the host;
 - every S_j lies below the exact sigma_j(A_c) (Rayleigh-Ritz) and the leading
   ones match it, sigma_j(A_c) following from the construction A = U Sigma V^T
   (eigenvalues of Sigma^2 - z z^T, z = Sigma U^T 1 / sqrt(m));
 - the Section 4 estimate of the residual is within 1.1 sigma_{k+1}(A_c).
"""
import numpy as np
import pytest

import synth as S
from gpu_util import cuda

pytestmark = pytest.mark.gpu


def _centred_spectrum(sigma, colsum, m, count):
    """sigma_1 .. sigma_count of A_c by bisection on the secular equation (FP64)."""
    d = np.asarray(sigma, dtype=np.float64) ** 2
    z2 = (np.asarray(sigma, dtype=np.float64) * colsum) ** 2 / m
    out = np.empty(count)
    for j in range(count):
        lo, hi = (d[j + 1] if j + 1 < d.size else 0.0), d[j]
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if mid <= lo or mid >= hi:
                break
            if 1.0 - np.sum(z2 / (d - mid)) > 0.0:
                lo = mid
            else:
                hi = mid
        out[j] = np.sqrt(0.5 * (lo + hi))
    return out


def test_precision_form_200000x20000_k200():
    torch = cuda()
    import paper_1412_3510_gb300 as rp
    w = S.WORKLOADS["dense_200000x20000_k200"]
    m, n, k, l, its = w["m"], w["n"], w["k"], w["l"], w["its"]
    sigma = w["spectrum"](min(m, n))
    A, colsum = S.haar_dense_torch(m, n, sigma, w["seed"], return_colsum=True)
    U, Sg, V = rp.rpca_dense(A, k, l, its=its, raw=False, seed=1, precision="bf16x3")
    torch.cuda.synchronize()

    Ud, Vd = U.double(), V.double()
    eye = torch.eye(k, dtype=torch.float64, device="cuda")
    assert torch.linalg.matrix_norm(Ud.T @ Ud - eye, 2).item() < 1e-4
    assert torch.linalg.matrix_norm(Vd.T @ Vd - eye, 2).item() < 1e-4
    s = Sg.double().cpu().numpy()
    assert np.all(np.diff(s) <= 0) and s[-1] > 0

    # S against the exact spectrum of A_c
    exact = _centred_spectrum(sigma, colsum, m, k + 1)
    assert np.all(s <= exact[:k] * (1 + 1e-5) + 1e-6 * exact[0])
    assert np.all(np.abs(s[:150] - exact[:150]) <= 1e-4 * exact[:150] + 1e-6 * exact[0])

    # A_c^T U = V diag(S) on sampled columns (FP64 on the host)
    rng = np.random.default_rng(7)
    cols = rng.choice(n, 8, replace=False)
    Uh = Ud.cpu().numpy()
    Vh = V.double().cpu().numpy()
    for j in cols:
        a = A[:, int(j)].double().cpu().numpy()
        ac = a - a.mean()
        lhs = ac @ Uh
        rhs = Vh[j] * s
        assert np.max(np.abs(lhs - rhs)) <= 1e-4 * np.linalg.norm(ac), (j, np.max(np.abs(lhs - rhs)))

    # residual within 1.1 sigma_{k+1}
    est = rp.rpca_resid_norm(A, U, Sg, V, iters=20, seed=7)
    assert est <= 1.1 * exact[k], (est, exact[k])

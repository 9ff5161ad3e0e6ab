"""Host-side helpers of bench.py that produce reference numbers (CPU)."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_sigma_k1_secular_matches_svd_of_centred_matrix():
    rng = np.random.default_rng(3)
    m, n = 700, 60
    U, _ = np.linalg.qr(rng.standard_normal((m, n)) + 0.3)       # columns with nonzero sums
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    sigma = np.exp(-np.arange(1, n + 1) / 10.0)
    A = (U * sigma) @ V.T
    Ac = A - A.mean(0)
    s = np.linalg.svd(Ac, compute_uv=False)
    for k in (0, 5, 17, n - 3):
        got = bench.sigma_k1_secular(sigma, U.sum(0), m, k)
        assert abs(got - s[k]) <= 1e-10 * s[0], (k, got, s[k])

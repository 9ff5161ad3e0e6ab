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


def test_split_bf16_roofline_bound():
    """HBM-bound at l = 102 (N = 112), tensor-bound at l = 210 (N = 224) on the measured peaks;
    fractions from the pass time by the stated formulas."""
    pk = {"hbm_gbs": 6748.0, "bf16_tflops": 1925.8, "bf16_tflops_sustained": 1725.8, "source": "measured"}
    m, n, l = 100000, 2000, 102
    pb = 4.0 * m * n + 4.0 * (m + n) * l
    r = bench.split_bf16_roofline(m, n, l, pb, 0.165, pk)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert abs(r["achieved"] - pb / 0.165e-3 / 1e9) < 1e-6 * r["achieved"]
    assert abs(r["tensor_frac"] - 6.0 * m * n * 112 / 0.165e-3 / 1e12 / 1725.8) < 1e-9
    m, n, l = 200000, 20000, 210
    pb = 4.0 * m * n + 4.0 * (m + n) * l
    r = bench.split_bf16_roofline(m, n, l, pb, 5.0, pk)
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert abs(r["achieved"] - 6.0 * m * n * 224 / 5e-3 / 1e12) < 1e-6 * r["achieved"]
    assert abs(r["frac"] - r["achieved"] / 1725.8) < 1e-12


def test_traffic_only_for_the_captured_kernel_and_workload(tmp_path, monkeypatch):
    """profiles/traffic.json entries apply to one kernel source (hash) and one workload."""
    import json
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(
        {"k": {"src_sha": "abc", "traffic_bytes_per_launch": 5.0, "workload": "w1"},
         "k2": {"src_sha": "def", "traffic_bytes_per_launch": 7.0}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_from_profiles("k", "abc", "w1") == 5.0
    assert bench.traffic_from_profiles("k", "abc", "w2") is None      # another workload
    assert bench.traffic_from_profiles("k", "xyz", "w1") is None      # the kernel changed
    assert bench.traffic_from_profiles("k2", "def", "any") == 7.0     # no workload named
    assert bench.traffic_from_profiles("missing", "abc", "w1") is None

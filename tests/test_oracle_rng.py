"""Pins for the oracle's random test matrix (Section 2: i.i.d. N(0,1) test vectors).

The Philox4x64-10 stream is checked word for word against numpy's own Philox
bit generator (an independent library implementation of the same published
generator); the Box-Muller normals are checked against the normal law with
scipy's Kolmogorov-Smirnov test and the first four moments.
"""
import numpy as np
import pytest
from scipy import stats

import oracle as O


def _numpy_blocks(key0, key1, first, count):
    # numpy's Philox increments the 256-bit counter before each block, so a
    # generator started at counter c yields the blocks for c+1, c+2, ...
    start = first - 1 if first > 0 else (1 << 256) - 1
    bg = np.random.Philox(counter=start, key=[key0, key1])
    return bg.random_raw(4 * count).reshape(count, 4)


@pytest.mark.parametrize("key", [(0, 0), (7, 0), (1234, 1), (2**64 - 1, 2**63 + 5)])
@pytest.mark.parametrize("first", [0, 1, 1000, 2**40 + 3])
def test_philox_matches_numpy(key, first):
    count = 257
    ctr = np.zeros((count, 4), dtype=np.uint64)
    ctr[:, 0] = np.arange(first, first + count, dtype=np.uint64)
    ours = O.philox4x64_10(ctr, *key)
    ref = _numpy_blocks(key[0], key[1], first, count)
    assert np.array_equal(ours, ref)


def test_philox_high_counter_words():
    # counters with the upper words set (numpy carries into them on overflow)
    bg = np.random.Philox(counter=(5 << 64) + (9 << 128) - 1, key=[11, 12])
    ref = bg.random_raw(4).reshape(1, 4)
    ctr = np.array([[0, 5, 9, 0]], dtype=np.uint64)
    assert np.array_equal(O.philox4x64_10(ctr, 11, 12), ref)


def test_uniform23_open_interval_and_exact():
    w = np.array([0, 2**64 - 1, 1 << 41, (1 << 41) - 1], dtype=np.uint64)
    u = O.uniform23(w)
    assert u[0] == 0.5 * 2.0**-23
    assert u[1] == 1.0 - 0.5 * 2.0**-23
    assert u[2] == 1.5 * 2.0**-23
    assert u[3] == u[0]
    assert np.all((u > 0) & (u < 1))
    # exactly representable in FP32, so both sides of the parity start from the same u
    assert np.array_equal(u.astype(np.float32).astype(np.float64), u)


def test_gaussian_omega_is_standard_normal():
    z = O.gaussian_omega(50000, 4, seed=99).ravel()
    assert abs(z.mean()) < 0.01
    assert abs(z.var() - 1.0) < 0.01
    assert abs(stats.skew(z)) < 0.03
    assert abs(stats.kurtosis(z)) < 0.06
    assert stats.kstest(z, "norm").pvalue > 1e-3


def test_gaussian_omega_layout_and_streams():
    a = O.gaussian_omega(33, 7, seed=5)
    b = O.gaussian_omega(7, 33, seed=5)
    # same element stream, different shapes: entry e = i*l + j
    assert np.array_equal(a.ravel(), b.ravel())
    c = O.gaussian_omega(33, 7, seed=5, stream=1)
    d = O.gaussian_omega(33, 7, seed=6)
    assert not np.allclose(a, c) and not np.allclose(a, d)
    # Box-Muller pairs: elements 4b, 4b+1 share a radius
    w = O.philox4x64_10(np.array([[0, 0, 0, 0]], dtype=np.uint64), 5, 0)
    u = O.uniform23(w)[0]
    r = np.sqrt(-2 * np.log(u[0]))
    assert np.isclose(np.hypot(a.ravel()[0], a.ravel()[1]), r, rtol=1e-14)
    assert np.isclose(np.arctan2(a.ravel()[1], a.ravel()[0]) % (2 * np.pi), 2 * np.pi * u[1], rtol=1e-12)

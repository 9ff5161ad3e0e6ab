"""Parity of the CUDA test-matrix generator (Section 2) with the oracle's."""
import numpy as np
import pytest

import oracle as O
from gpu_util import cuda, to_np

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("key", [(0, 0), (1234, 1), (2**64 - 1, 7)])
@pytest.mark.parametrize("first,count", [(0, 1), (0, 1000), (2**40 + 3, 333)])
def test_philox_words_bit_exact(key, first, count):
    cuda()
    import paper_1412_3510_gb300 as rp
    g = rp.rpca_philox4x64_10(key[0], key[1], first, count).cpu().numpy().view(np.uint64)
    ctr = np.zeros((count, 4), dtype=np.uint64)
    ctr[:, 0] = np.arange(first, first + count, dtype=np.uint64)
    assert np.array_equal(g, O.philox4x64_10(ctr, *key))


@pytest.mark.parametrize("n,l,seed,stream", [(1, 1, 0, 0), (1000, 12, 7, 0), (2001, 102, 99, 0),
                                             (37, 5, 3, 1), (20000, 210, 1237, 0)])
def test_gaussian_omega_matches_oracle(n, l, seed, stream):
    cuda()
    import paper_1412_3510_gb300 as rp
    g = to_np(rp.rpca_gaussian_omega(n, l, seed, stream))
    o = O.gaussian_omega(n, l, seed, stream)
    # the uniforms are bit-identical; only FP32 log / sincos rounding differs
    assert np.allclose(g, o, rtol=2e-6, atol=2e-6), np.max(np.abs(g - o))

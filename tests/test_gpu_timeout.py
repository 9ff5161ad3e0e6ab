"""The bounded device-side waits: a wait whose arrival never comes ends with
RPCA_ERR_TIMEOUT in the status block, the GPU context stays usable, and the next
call runs normally (no fault or hang is provoked: the waited-on mbarrier simply
never receives its arrival, and nothing else is in flight)."""
import ctypes

import numpy as np
import pytest

from gpu_util import cuda, to_dev, to_np

pytestmark = pytest.mark.gpu


def test_wait_runs_out_and_reports_timeout():
    torch = cuda()
    import paper_1412_3510_gb300 as rp
    from paper_1412_3510_gb300 import _lib
    lib = _lib.load()
    ws = rp.workspace(512, "cuda")
    for limit in (20000, 2000000):
        waited = ctypes.c_int64(0)
        code = lib.rpca_wait_selftest(limit, ctypes.byref(waited), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert code == 0
        assert rp.rpca_read_status(ws) == _lib.RPCA_ERR_TIMEOUT
        assert rp.read_status_block(ws)["timeouts"] == 1
        assert limit <= waited.value < limit + 1000000          # gave up right after the limit
    # the context is intact: an ordinary PCA runs and is correct
    import oracle as O
    import synth as S_
    A = S_.haar_dense_np(300, 200, np.exp(-np.arange(1, 201) / 5.0), seed=3)
    U, S, V = rp.rpca_dense(to_dev(A), 5, 7, its=2, raw=True, seed=1)
    _, ref, _ = O.rpca(A, 5, 7, 2, raw=True, seed=1)
    assert np.all(np.abs(to_np(S) - ref) <= 1e-4 * ref + 1e-6 * ref[0])


def test_wait_selftest_rejects_bad_arguments():
    torch = cuda()
    import paper_1412_3510_gb300 as rp
    from paper_1412_3510_gb300 import _lib
    lib = _lib.load()
    ws = rp.workspace(512, "cuda")
    waited = ctypes.c_int64(0)
    assert lib.rpca_wait_selftest(10, ctypes.byref(waited), ctypes.c_void_p(ws.data_ptr()), 512, None) == \
        _lib.RPCA_ERR_INVALID_ARG
    assert lib.rpca_wait_selftest(10000, ctypes.byref(waited), ctypes.c_void_p(ws.data_ptr()), 100, None) == \
        _lib.RPCA_ERR_WORKSPACE

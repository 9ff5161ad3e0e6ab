"""rpca_dense_pass_noalloc: the product for callers that cannot allocate device memory.

It takes no workspace (its scratch is a fixed buffer inside the library), so
callers that get all device memory from a host framework's pool, or that must
not pay cudaMalloc's synchronisation, can still run a pass.  Its results must
match rpca_dense_pass (which takes a caller workspace) exactly: both run the
same deterministic kernels on the same inputs, so any difference would come
from the shared buffer.  Two rounds of calls in a row check that its leftover
contents from the previous call do not leak into the next.
"""
import ctypes

import numpy as np
import pytest

from paper_1412_3510_gb300 import _lib

CASES = [  # m, n, w, adjoint, precision
    (300, 200, 16, False, "fp32"),
    (300, 200, 16, True, "fp32"),
    (1000, 333, 104, False, "bf16x3"),
    (1000, 333, 104, True, "bf16x3"),
    (4097, 130, 112, True, "bf16x3"),
]


def _call_noalloc(A, B, adjoint, precision):
    import torch
    lib = _lib.load()
    m, n = A.shape
    w = B.shape[1]
    C = torch.full((n if adjoint else m, w), float("nan"), device="cuda")
    code = lib.rpca_dense_pass_noalloc(ctypes.c_void_p(A.data_ptr()), m, n, A.stride(0), int(adjoint),
                                       ctypes.c_void_p(B.data_ptr()), w, ctypes.c_void_p(C.data_ptr()),
                                       _lib.PREC[precision],
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return code, C


@pytest.mark.gpu
def test_noalloc_matches_workspace_entry_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1412_3510_gb300 as rp
    for rnd in range(2):
        for m, n, w, adjoint, precision in CASES:
            rng = np.random.default_rng(1000 * rnd + m + w)
            A = torch.from_numpy(rng.standard_normal((m, n)).astype(np.float32)).cuda()
            B = torch.from_numpy(rng.standard_normal((m if adjoint else n, w)).astype(np.float32)).cuda()
            ref = rp.rpca_dense_pass(A, B, adjoint=adjoint, precision=precision)
            code, C = _call_noalloc(A, B, adjoint, precision)
            assert code == 0, _lib.load().rpca_status_string(code)
            torch.cuda.synchronize()
            assert torch.equal(C, ref), (rnd, m, n, w, adjoint, precision)


def test_noalloc_rejects_problems_larger_than_its_buffer():
    # host-side check, before any device work: needs no GPU
    lib = _lib.load()
    m, n, w = 2_000_000, 4000, 256
    need = lib.rpca_dense_pass_workspace_size(m, n, w, 1, _lib.PREC["bf16x3"])
    assert need > _lib.RPCA_NOALLOC_SCRATCH_BYTES
    fake = ctypes.c_void_p(256)
    code = lib.rpca_dense_pass_noalloc(fake, m, n, n, 1, fake, w, fake, _lib.PREC["bf16x3"], None)
    assert code == _lib.RPCA_ERR_WORKSPACE

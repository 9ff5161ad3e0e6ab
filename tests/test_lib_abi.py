"""The C-ABI library loads and exports every entry point include/rpca.h declares (no GPU needed)."""
import ctypes
import os

import pytest

from paper_1412_3510_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(_lib.LIB_PATH):
        from paper_1412_3510_gb300 import build
        build.build()
    return ctypes.CDLL(_lib.LIB_PATH)


def test_exports_every_declared_symbol(lib):
    names = _lib.header_symbols()
    assert "rpca_dense" in names and "rpca_csr" in names and "rpca_resid_norm" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, f"declared in rpca.h but not exported: {missing}"


def test_binding_declares_every_header_symbol():
    declared = {name for name, _, _ in _lib.SIGNATURES}
    assert set(_lib.header_symbols()) <= declared


def test_host_only_entry_points(lib):
    L = _lib.load()
    assert L.rpca_status_string(0) == b"ok"
    assert L.rpca_status_string(-2).startswith(b"workspace")
    o = _lib.RpcaOpts()
    L.rpca_default_opts(ctypes.byref(o), 10)
    assert (o.k, o.l, o.its, o.raw) == (10, 12, 2, 0)
    # workspace query is pure host arithmetic
    assert L.rpca_dense_workspace_size(2000, 1000, ctypes.byref(o)) > 0
    bad = _lib.RpcaOpts()
    L.rpca_default_opts(ctypes.byref(bad), 300)          # l = 302 > RPCA_MAX_L
    assert L.rpca_dense_workspace_size(2000, 1000, ctypes.byref(bad)) == 0


def test_argument_errors_need_no_gpu(lib):
    L = _lib.load()
    o = _lib.RpcaOpts()
    L.rpca_default_opts(ctypes.byref(o), 5)
    # null A / outputs are rejected before anything touches the device
    assert L.rpca_dense(None, 100, 50, 50, ctypes.byref(o), None, 5, None, None, 5, None, 0, None) == _lib.RPCA_ERR_INVALID_ARG
    o.l = 3   # l < k
    fake = ctypes.c_void_p(256)
    assert L.rpca_dense(fake, 100, 50, 50, ctypes.byref(o), fake, 5, fake, fake, 5, fake, 1 << 30, None) == _lib.RPCA_ERR_INVALID_ARG
    o.l = 7
    assert L.rpca_dense(fake, 100, 50, 49, ctypes.byref(o), fake, 5, fake, fake, 5, fake, 1 << 30, None) == _lib.RPCA_ERR_INVALID_ARG
    # misaligned or short workspace
    assert L.rpca_dense(fake, 100, 50, 50, ctypes.byref(o), fake, 5, fake, fake, 5, ctypes.c_void_p(257), 1 << 30, None) == _lib.RPCA_ERR_WORKSPACE
    assert L.rpca_dense(fake, 100, 50, 50, ctypes.byref(o), fake, 5, fake, fake, 5, fake, 16, None) == _lib.RPCA_ERR_WORKSPACE


def test_option_errors_need_no_gpu(lib):
    L = _lib.load()
    fake = ctypes.c_void_p(256)
    o = _lib.RpcaOpts()
    L.rpca_default_opts(ctypes.byref(o), 150)
    o.l = 170
    o.renorm = 1                      # the LU renormalisation holds 2l x (l + 1) per node: l <= 160
    args = (fake, 4000, 1000, 1000, ctypes.byref(o), fake, 150, fake, fake, 150, fake, 1 << 40, None)
    assert L.rpca_dense(*args) == _lib.RPCA_ERR_UNSUPPORTED
    o.renorm = 2                      # not a renormalisation
    assert L.rpca_dense(*args) == _lib.RPCA_ERR_INVALID_ARG
    o.renorm = 0
    o.precision = 5                   # not a precision
    assert L.rpca_dense(*args) == _lib.RPCA_ERR_INVALID_ARG

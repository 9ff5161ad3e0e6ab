"""ctypes loader for librpca.so (declarations mirror include/rpca.h)."""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librpca.so")

RPCA_OK = 0
RPCA_FELL_BACK = 1
RPCA_ERR_INVALID_ARG = -1
RPCA_ERR_WORKSPACE = -2
RPCA_ERR_CUDA = -3
RPCA_ERR_NONFINITE = -4
RPCA_ERR_BREAKDOWN = -5
RPCA_ERR_TIMEOUT = -6
RPCA_ERR_UNSUPPORTED = -7
RPCA_MAX_L = 224
RPCA_NOALLOC_SCRATCH_BYTES = 64 << 20
RPCA_MLP_FEATURES = 16
RPCA_MLP_HIDDEN = 128
RPCA_MLP_PARAMS = 18817
RPCA_MLP_PACKED_BYTES = 38416

PREC = {"fp32": 0, "bf16x3": 1}
RENORM = {"cholqr": 0, "lu": 1}
RPCA_RENORM_ODD_ONLY = 4
RPCA_PREC_SMALL_FP64 = 16


class RpcaOpts(C.Structure):
    _fields_ = [
        ("k", C.c_int32), ("l", C.c_int32), ("its", C.c_int32), ("raw", C.c_int32),
        ("seed", C.c_uint64), ("precision", C.c_int32), ("renorm", C.c_int32),
        ("omega", C.c_void_p), ("col_weights", C.c_void_p),
    ]


# (name, restype, argtypes) for every symbol include/rpca.h declares
_I64, _I32, _U64, _P, _SZ = C.c_int64, C.c_int32, C.c_uint64, C.c_void_p, C.c_size_t
_OPTS = C.POINTER(RpcaOpts)
SIGNATURES = [
    ("rpca_default_opts", None, [_OPTS, _I32]),
    ("rpca_dense_workspace_size", _SZ, [_I64, _I64, _OPTS]),
    ("rpca_dense", C.c_int, [_P, _I64, _I64, _I64, _OPTS, _P, _I64, _P, _P, _I64, _P, _SZ, _P]),
    ("rpca_sym_workspace_size", _SZ, [_I64, _OPTS]),
    ("rpca_sym", C.c_int, [_P, _I64, _I64, _OPTS, _P, _I64, _P, _P, _I64, _P, _SZ, _P]),
    ("rpca_nystrom", C.c_int, [_P, _I64, _I64, _OPTS, _P, _I64, _P, _P, _SZ, _P]),
    ("rpca_csr_workspace_size", _SZ, [_I64, _I64, _I64, _OPTS]),
    ("rpca_csr", C.c_int, [_I64, _I64, _I64, _P, _P, _P, _OPTS, _P, _I64, _P, _P, _I64, _P, _SZ, _P]),
    ("rpca_resid_workspace_size", _SZ, [_I64, _I64, _I32]),
    ("rpca_resid_norm", C.c_int, [_P, _I64, _I64, _I64, _I32, _P, _I64, _P, _P, _I64, _I32, _I32, _U64,
                                  _P, _P, _SZ, _P]),
    ("rpca_dense_pass_workspace_size", _SZ, [_I64, _I64, _I32, _I32, _I32]),
    ("rpca_dense_pass", C.c_int, [_P, _I64, _I64, _I64, _I32, _P, _I32, _P, _I32, _P, _SZ, _P]),
    ("rpca_dense_pass_noalloc", C.c_int, [_P, _I64, _I64, _I64, _I32, _P, _I32, _P, _I32, _P]),
    ("rpca_resid_csr_workspace_size", _SZ, [_I64, _I64, _I64, _I32]),
    ("rpca_resid_norm_csr", C.c_int, [_I64, _I64, _I64, _P, _P, _P, _I32, _P, _I64, _P, _P, _I64, _I32, _I32, _U64,
                                      _P, _P, _SZ, _P]),
    ("rpca_batched_workspace_size", _SZ, [_I32, _I64, _I64, _OPTS]),
    ("rpca_batched", C.c_int, [_I32, _P, _I64, _I64, _OPTS, _P, _P, _P, _SZ, _P]),
    ("rpca_batched_tune", C.c_int, [_I32, _P, _I64, _I64, _OPTS, _P, _P, _P, _SZ, _P, C.POINTER(C.c_int32),
                                    C.POINTER(C.c_int32), C.POINTER(C.c_float)]),
    ("rpca_batched_learned_workspace_size", _SZ, [_I32, _I64, _I64, _OPTS]),
    ("rpca_batched_learned", C.c_int, [_I32, _P, _I64, _I64, _OPTS, _P, _I32, C.c_float, _P, _P, _P, _SZ, _P]),
    ("rpca_features_workspace_size", _SZ, [_I64, _I64]),
    ("rpca_sketch_features", C.c_int, [_P, _I64, _I64, _I64, _I32, _U64, _P, _P, _SZ, _P]),
    ("rpca_batched_features_workspace_size", _SZ, [_I64]),
    ("rpca_batched_features", C.c_int, [_I32, _P, _I64, _I32, _U64, _P, _P, _P, _SZ, _P]),
    ("rpca_mlp_pack", C.c_int, [_P, _P, _P]),
    ("rpca_mlp_forward_workspace_size", _SZ, []),
    ("rpca_mlp_forward", C.c_int, [_P, _P, _I64, _P, _P, _P, _SZ, _P]),
    ("rpca_mlp_grad_workspace_size", _SZ, [_I64]),
    ("rpca_mlp_loss_grad", C.c_int, [_P, _P, _P, _I64, _P, _P, _P, _SZ, _P]),
    ("rpca_mlp_adam", C.c_int, [_P, _P, _P, _P, _I32, C.c_float, C.c_float, C.c_float, C.c_float, _P]),
    ("rpca_leverage_target", C.c_int, [_P, _I64, _I64, _I32, _P, _P]),
    ("rpca_dense_learned_workspace_size", _SZ, [_I64, _I64, _OPTS]),
    ("rpca_dense_learned", C.c_int, [_P, _I64, _I64, _I64, _OPTS, _P, _I32, C.c_double, _P, _I64, _P, _P, _I64,
                                     C.POINTER(C.c_double), _P, _SZ, _P]),
    ("rpca_small_svd_workspace_size", _SZ, [_I32]),
    ("rpca_small_svd", C.c_int, [_P, _I32, _P, _P, _P, _P, _SZ, _P]),
    ("rpca_gaussian_omega", C.c_int, [_I64, _I32, _U64, _U64, _P, _I64, _P]),
    ("rpca_philox4x64_10", C.c_int, [_U64, _U64, _U64, _I64, _P, _P]),
    ("rpca_wait_selftest", C.c_int, [_I64, C.POINTER(C.c_int64), _P, _SZ, _P]),
    ("rpca_read_status", C.c_int, [_P, _P, C.POINTER(C.c_int32)]),
    ("rpca_status_string", C.c_char_p, [C.c_int]),
    ("rpca_launch_count", C.c_int64, []),
    ("rpca_timing_enable", C.c_int, [_I32]),
    ("rpca_timing_select", C.c_int, [C.c_uint32]),
    ("rpca_timing_reset", C.c_int, []),
    ("rpca_timing_read", C.c_int, [_I32, C.POINTER(C.c_int64), C.POINTER(C.c_double)]),
]

_lib = None


def header_symbols() -> list[str]:
    """Every function name declared in include/rpca.h (parsed from the header text)."""
    import re
    path = os.path.join(os.path.dirname(_HERE), "include", "rpca.h")
    with open(path) as f:
        text = f.read()
    return sorted(set(re.findall(r"\b(rpca_[a-z0-9_]+)\s*\(", text)))


def load(path: str = LIB_PATH):
    """Load librpca.so and declare its signatures; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} is missing: build the CUDA library first "
            "(python -c 'import __graft_entry__ as g; g.build()'); there is no CPU fallback")
    lib = C.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name, None)
        if fn is None:
            continue
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib

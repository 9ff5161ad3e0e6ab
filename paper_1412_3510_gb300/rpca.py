"""Python binding of librpca.so: the C-ABI entry points under the same names.

Argument marshalling only.  Every step of the method runs in the library's CUDA
kernels; PyTorch supplies device memory (outputs, workspace) and the current
stream.  Nothing here computes, and there is no CPU fallback: a missing
library or a CPU tensor raises.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib as L


class RpcaError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        lib = L.load()
        msg = lib.rpca_status_string(code).decode()
        super().__init__(f"{what}: {msg} (status {code})" if what else f"{msg} (status {code})")
        self.code = code


def _check(code: int, what: str) -> int:
    if code < 0:
        raise RpcaError(code, what)
    return code


def _ptr(t):
    return C.c_void_p(0 if t is None else t.data_ptr())


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _need_cuda(t: torch.Tensor, name: str, dtype=torch.float32):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}")


def _rowmajor_ld(t: torch.Tensor, name: str) -> int:
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError(f"{name} must be 2-D with unit column stride (row-major)")
    return max(t.stride(0), t.shape[1])


def make_opts(k, l=None, its=2, raw=False, seed=0, precision="fp32", renorm="cholqr",
              omega=None, col_weights=None, odd_only=False, small_fp64=False) -> L.RpcaOpts:
    o = L.RpcaOpts()
    o.k = int(k)
    o.l = int(k + 2 if l is None else l)
    o.its = int(its)
    o.raw = int(bool(raw))
    o.seed = int(seed) & ((1 << 64) - 1)
    o.precision = L.PREC[precision] | (L.RPCA_PREC_SMALL_FP64 if small_fp64 else 0)
    o.renorm = L.RENORM[renorm] | (L.RPCA_RENORM_ODD_ONLY if odd_only else 0)
    o.omega = None if omega is None else omega.data_ptr()
    o.col_weights = None if col_weights is None else col_weights.data_ptr()
    return o


def rpca_dense_workspace_size(m: int, n: int, opts: L.RpcaOpts) -> int:
    return int(L.load().rpca_dense_workspace_size(m, n, C.byref(opts)))


def workspace(nbytes: int, device) -> torch.Tensor:
    """A 256-byte-aligned device buffer of nbytes (torch allocations are 512-aligned)."""
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def rpca_dense(A: torch.Tensor, k: int, l: int | None = None, its: int = 2, raw: bool = False,
               seed: int = 0, precision: str = "fp32", renorm: str = "cholqr",
               omega: torch.Tensor | None = None, col_weights: torch.Tensor | None = None,
               ws: torch.Tensor | None = None, out=None, stream=None, check: bool = True,
               odd_only: bool = False, small_fp64: bool = False):
    """Randomized PCA A_c ~ U diag(S) V^T (Sections 2 and 5 of the paper).

    A: m x n float32 CUDA tensor, row-major (any leading dimension >= n).
    Returns (U m x k, S k, V n x k).  With check=True the device status word
    is read after the call (one stream synchronisation).
    """
    _need_cuda(A, "A")
    lda = _rowmajor_ld(A, "A")
    m, n = A.shape
    if omega is not None:
        _need_cuda(omega, "omega")
        omega = omega.contiguous()
    if col_weights is not None:
        _need_cuda(col_weights, "col_weights")
        col_weights = col_weights.contiguous()
    opts = make_opts(k, l, its, raw, seed, precision, renorm, omega, col_weights, odd_only, small_fp64)
    lib = L.load()
    need = rpca_dense_workspace_size(m, n, opts)
    if need == 0:
        raise RpcaError(L.RPCA_ERR_INVALID_ARG, "rpca_dense_workspace_size")
    if ws is None or ws.numel() < need:
        ws = workspace(need, A.device)
    if out is None:
        U = torch.empty(m, k, dtype=torch.float32, device=A.device)
        S = torch.empty(k, dtype=torch.float32, device=A.device)
        V = torch.empty(n, k, dtype=torch.float32, device=A.device)
    else:
        U, S, V = out
    ldu = _rowmajor_ld(U, "U")
    ldv = _rowmajor_ld(V, "V")
    st = _stream(stream)
    code = lib.rpca_dense(_ptr(A), m, n, lda, C.byref(opts), _ptr(U), ldu, _ptr(S), _ptr(V), ldv,
                          _ptr(ws), ws.numel(), st)
    _check(code, "rpca_dense")
    if check:
        status = rpca_read_status(ws, stream)
        _check(status, "rpca_dense (device)")
    return U, S, V


def _sym_call(A, k, l, its, seed, precision, renorm, omega, odd_only, ws, out, stream, check, nystrom,
              small_fp64=False):
    _need_cuda(A, "A")
    lda = _rowmajor_ld(A, "A")
    n = A.shape[0]
    if A.shape[1] != n:
        raise ValueError("A must be square")
    if omega is not None:
        _need_cuda(omega, "omega")
        omega = omega.contiguous()
    opts = make_opts(k, l, its, True, seed, precision, renorm, omega, None, odd_only, small_fp64)
    lib = L.load()
    need = int(lib.rpca_sym_workspace_size(n, C.byref(opts)))
    if need == 0:
        raise RpcaError(L.RPCA_ERR_INVALID_ARG, "rpca_sym_workspace_size")
    if ws is None or ws.numel() < need:
        ws = workspace(need, A.device)
    if out is None:
        U = torch.empty(n, k, dtype=torch.float32, device=A.device)
        S = torch.empty(k, dtype=torch.float32, device=A.device)
        V = None if nystrom else torch.empty(n, k, dtype=torch.float32, device=A.device)
    else:
        U, S, V = (tuple(out) + (None,))[:3]
    if nystrom:
        code = lib.rpca_nystrom(_ptr(A), n, lda, C.byref(opts), _ptr(U), _rowmajor_ld(U, "U"), _ptr(S), _ptr(ws),
                                ws.numel(), _stream(stream))
    else:
        code = lib.rpca_sym(_ptr(A), n, lda, C.byref(opts), _ptr(U), _rowmajor_ld(U, "U"), _ptr(S), _ptr(V),
                            _rowmajor_ld(V, "V"), _ptr(ws), ws.numel(), _stream(stream))
    name = "rpca_nystrom" if nystrom else "rpca_sym"
    _check(code, name)
    if check:
        _check(rpca_read_status(ws, stream), name + " (device)")
    return (U, S) if nystrom else (U, S, V)


def rpca_sym(A: torch.Tensor, k: int, l: int | None = None, its: int = 2, seed: int = 0,
             precision: str = "fp32", renorm: str = "cholqr", omega: torch.Tensor | None = None,
             odd_only: bool = False, ws: torch.Tensor | None = None, out=None, stream=None, check: bool = True,
             small_fp64: bool = False):
    """Self-adjoint A (n x n): Section 5's loop of products with A only, then
    B = Q^T A Q; returns (U, S, V) with A ~ U diag(S) V^T, V = U diag(sign(lambda))."""
    return _sym_call(A, k, l, its, seed, precision, renorm, omega, odd_only, ws, out, stream, check, False, small_fp64)


def rpca_nystrom(A: torch.Tensor, k: int, l: int | None = None, its: int = 2, seed: int = 0,
                 precision: str = "fp32", renorm: str = "cholqr", omega: torch.Tensor | None = None,
                 odd_only: bool = False, ws: torch.Tensor | None = None, out=None, stream=None,
                 check: bool = True, small_fp64: bool = False):
    """Stabilised Nystrom approximation of a nonnegative-definite A (Section 3):
    returns (U, S) with A ~ U diag(S) U^T."""
    return _sym_call(A, k, l, its, seed, precision, renorm, omega, odd_only, ws, out, stream, check, True, small_fp64)


def rpca_small_svd(M: torch.Tensor, stream=None):
    """SVD of a small FP64 matrix M (l x l, CUDA) as the FP64 l x l path computes it:
    returns (S, W, Z) with M = W diag(S) Z^T."""
    if not isinstance(M, torch.Tensor) or not M.is_cuda or M.dtype != torch.float64:
        raise ValueError("M must be a float64 CUDA tensor")
    l = int(M.shape[0])
    if M.dim() != 2 or M.shape[1] != l:
        raise ValueError("M must be square")
    M = M.contiguous()
    lib = L.load()
    need = int(lib.rpca_small_svd_workspace_size(l))
    if need == 0:
        raise RpcaError(L.RPCA_ERR_INVALID_ARG, "rpca_small_svd_workspace_size")
    ws = workspace(need, M.device)
    S = torch.empty(l, dtype=torch.float64, device=M.device)
    W = torch.empty(l, l, dtype=torch.float64, device=M.device)
    Z = torch.empty(l, l, dtype=torch.float64, device=M.device)
    _check(lib.rpca_small_svd(_ptr(M), l, _ptr(S), _ptr(W), _ptr(Z), _ptr(ws), ws.numel(), _stream(stream)),
           "rpca_small_svd")
    _check(rpca_read_status(ws, stream), "rpca_small_svd (device)")
    return S, W, Z


def rpca_read_status(ws: torch.Tensor, stream=None) -> int:
    out = C.c_int32(0)
    _check(L.load().rpca_read_status(_ptr(ws), _stream(stream), C.byref(out)), "rpca_read_status")
    return int(out.value)


def read_status_block(ws: torch.Tensor) -> dict:
    """The device status block's counters (shifts, Jacobi sweeps...) after a synchronisation."""
    torch.cuda.current_stream(ws.device).synchronize()
    v = ws[:256].view(torch.int32).cpu().tolist()
    return {"status": v[0], "flags": v[1], "shifts": v[2], "jacobi_sweeps": v[3],
            "jacobi_unconverged": v[4], "timeouts": v[5]}


def rpca_gaussian_omega(n: int, l: int, seed: int, stream_id: int = 0, device="cuda", stream=None):
    out = torch.empty(n, l, dtype=torch.float32, device=device)
    _check(L.load().rpca_gaussian_omega(n, l, seed & ((1 << 64) - 1), stream_id, _ptr(out), l,
                                        _stream(stream)), "rpca_gaussian_omega")
    return out


def rpca_philox4x64_10(key0: int, key1: int, first: int, nblocks: int, device="cuda", stream=None):
    out = torch.empty(nblocks, 4, dtype=torch.int64, device=device)
    m64 = (1 << 64) - 1
    _check(L.load().rpca_philox4x64_10(key0 & m64, key1 & m64, first & m64, nblocks, _ptr(out),
                                       _stream(stream)), "rpca_philox4x64_10")
    return out


def rpca_launch_count() -> int:
    return int(L.load().rpca_launch_count())


def rpca_resid_norm(A: torch.Tensor, U: torch.Tensor, S: torch.Tensor, V: torch.Tensor,
                    raw: bool = False, iters: int = 20, seed: int = 0, ws: torch.Tensor | None = None,
                    est: torch.Tensor | None = None, stream=None, sync: bool = True):
    """Power-method estimate of ||A_c - U diag(S) V^T||_2 (Section 4), as a float (sync=True)
    or as the 1-element float64 device tensor it is written to (sync=False)."""
    _need_cuda(A, "A")
    lda = _rowmajor_ld(A, "A")
    m, n = A.shape
    k = int(S.numel())
    lib = L.load()
    need = int(lib.rpca_resid_workspace_size(m, n, k))
    if need == 0:
        raise RpcaError(L.RPCA_ERR_INVALID_ARG, "rpca_resid_workspace_size")
    if ws is None or ws.numel() < need:
        ws = workspace(need, A.device)
    if est is None:
        est = torch.empty(1, dtype=torch.float64, device=A.device)
    ldu = _rowmajor_ld(U, "U") if k else k
    ldv = _rowmajor_ld(V, "V") if k else k
    code = lib.rpca_resid_norm(_ptr(A), m, n, lda, int(bool(raw)), _ptr(U), ldu, _ptr(S), _ptr(V), ldv,
                               k, int(iters), seed & ((1 << 64) - 1), _ptr(est), _ptr(ws), ws.numel(),
                               _stream(stream))
    _check(code, "rpca_resid_norm")
    if sync:
        _check(rpca_read_status(ws, stream), "rpca_resid_norm (device)")
        return float(est.item())
    return est


def rpca_timing_enable(on: bool = True, reserve: int = 0) -> None:
    """Turn stage timing on or off; `reserve` events are created up front."""
    _check(L.load().rpca_timing_enable(max(int(bool(on)), int(reserve) if on else 0)), "rpca_timing_enable")


def rpca_timing_select(kinds=None) -> None:
    """Time only the given stage kinds (None: all)."""
    mask = 0xFFFFFFFF if kinds is None else sum(1 << int(k) for k in kinds)
    _check(L.load().rpca_timing_select(mask), "rpca_timing_select")


def rpca_timing_reset() -> None:
    _check(L.load().rpca_timing_reset(), "rpca_timing_reset")


def rpca_timing_read(kind: int):
    """(launches, total milliseconds) of the timed stage `kind` since the last reset."""
    c = C.c_int64(0)
    t = C.c_double(0.0)
    _check(L.load().rpca_timing_read(int(kind), C.byref(c), C.byref(t)), "rpca_timing_read")
    return int(c.value), float(t.value)


def rpca_dense_pass(A: torch.Tensor, B: torch.Tensor, adjoint: bool = False, precision: str = "fp32",
                    ws: torch.Tensor | None = None, out: torch.Tensor | None = None, stream=None,
                    check: bool = True):
    """One product without centring: A @ B (adjoint=False) or A.T @ B (adjoint=True).

    B: (n or m) x w float32 CUDA, contiguous, w a multiple of 8 (<= 256)."""
    _need_cuda(A, "A")
    _need_cuda(B, "B")
    lda = _rowmajor_ld(A, "A")
    m, n = A.shape
    B = B.contiguous()
    w = int(B.shape[1])
    lib = L.load()
    need = int(lib.rpca_dense_pass_workspace_size(m, n, w, int(adjoint), L.PREC[precision]))
    if need == 0:
        raise RpcaError(L.RPCA_ERR_INVALID_ARG, "rpca_dense_pass_workspace_size")
    if ws is None or ws.numel() < need:
        ws = workspace(need, A.device)
    rows = n if adjoint else m
    C = torch.empty(rows, w, dtype=torch.float32, device=A.device) if out is None else out
    code = lib.rpca_dense_pass(_ptr(A), m, n, lda, int(adjoint), _ptr(B), w, _ptr(C), L.PREC[precision],
                               _ptr(ws), ws.numel(), _stream(stream))
    _check(code, "rpca_dense_pass")
    if check:
        _check(rpca_read_status(ws, stream), "rpca_dense_pass (device)")
    return C


def _need_i32(t, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.int32:
        raise ValueError(f"{name} must be an int32 CUDA tensor")


def rpca_csr(row_ptr: torch.Tensor, col_idx: torch.Tensor, val: torch.Tensor, shape, k: int,
             l: int | None = None, its: int = 2, raw: bool = False, seed: int = 0,
             omega: torch.Tensor | None = None, col_weights: torch.Tensor | None = None,
             ws: torch.Tensor | None = None, out=None, stream=None, check: bool = True,
             renorm: str = "cholqr", odd_only: bool = False, small_fp64: bool = False):
    """Randomized PCA of a CSR matrix (row_ptr int32 m+1, col_idx int32 nnz, val float32 nnz)."""
    m, n = int(shape[0]), int(shape[1])
    _need_i32(row_ptr, "row_ptr")
    _need_i32(col_idx, "col_idx")
    _need_cuda(val, "val")
    nnz = int(val.numel())
    if omega is not None:
        _need_cuda(omega, "omega")
        omega = omega.contiguous()
    if col_weights is not None:
        _need_cuda(col_weights, "col_weights")
        col_weights = col_weights.contiguous()
    opts = make_opts(k, l, its, raw, seed, "fp32", renorm, omega, col_weights, odd_only, small_fp64)
    lib = L.load()
    need = int(lib.rpca_csr_workspace_size(m, n, nnz, C.byref(opts)))
    if need == 0:
        raise RpcaError(L.RPCA_ERR_INVALID_ARG, "rpca_csr_workspace_size")
    if ws is None or ws.numel() < need:
        ws = workspace(need, val.device)
    if out is None:
        U = torch.empty(m, k, dtype=torch.float32, device=val.device)
        S = torch.empty(k, dtype=torch.float32, device=val.device)
        V = torch.empty(n, k, dtype=torch.float32, device=val.device)
    else:
        U, S, V = out
    code = lib.rpca_csr(m, n, nnz, _ptr(row_ptr), _ptr(col_idx), _ptr(val), C.byref(opts), _ptr(U),
                        _rowmajor_ld(U, "U"), _ptr(S), _ptr(V), _rowmajor_ld(V, "V"), _ptr(ws), ws.numel(),
                        _stream(stream))
    _check(code, "rpca_csr")
    if check:
        _check(rpca_read_status(ws, stream), "rpca_csr (device)")
    return U, S, V


def rpca_resid_norm_csr(row_ptr, col_idx, val, shape, U, S, V, raw: bool = False, iters: int = 20,
                        seed: int = 0, ws=None, est=None, stream=None, sync: bool = True):
    """Section 4 residual estimate for a CSR matrix."""
    m, n = int(shape[0]), int(shape[1])
    nnz = int(val.numel())
    k = int(S.numel())
    lib = L.load()
    need = int(lib.rpca_resid_csr_workspace_size(m, n, nnz, k))
    if need == 0:
        raise RpcaError(L.RPCA_ERR_INVALID_ARG, "rpca_resid_csr_workspace_size")
    if ws is None or ws.numel() < need:
        ws = workspace(need, val.device)
    if est is None:
        est = torch.empty(1, dtype=torch.float64, device=val.device)
    ldu = _rowmajor_ld(U, "U") if k else k
    ldv = _rowmajor_ld(V, "V") if k else k
    code = lib.rpca_resid_norm_csr(m, n, nnz, _ptr(row_ptr), _ptr(col_idx), _ptr(val), int(bool(raw)), _ptr(U),
                                   ldu, _ptr(S), _ptr(V), ldv, k, int(iters), seed & ((1 << 64) - 1), _ptr(est),
                                   _ptr(ws), ws.numel(), _stream(stream))
    _check(code, "rpca_resid_norm_csr")
    if sync:
        _check(rpca_read_status(ws, stream), "rpca_resid_norm_csr (device)")
        return float(est.item())
    return est


class Batch:
    """Device-side descriptors for rpca_batched: one (A, U, S, V) per matrix.

    mats: list of m_i x n_i float32 CUDA tensors (row-major).  Outputs are
    allocated here (U_i m_i x k, S_i k, V_i n_i x k)."""

    def __init__(self, mats, k: int, device=None):
        device = device or mats[0].device
        self.mats = mats
        self.k = k
        # outputs as views of three contiguous buffers (one copy reads all of them back)
        mu = [int(a.shape[0]) * k for a in mats]
        nv = [int(a.shape[1]) * k for a in mats]
        self.U_all = torch.empty(sum(mu), dtype=torch.float32, device=device)
        self.S_all = torch.empty(len(mats) * k, dtype=torch.float32, device=device)
        self.V_all = torch.empty(sum(nv), dtype=torch.float32, device=device)
        self.U, self.S, self.V = [], [], []
        ou = ov = 0
        for i, a in enumerate(mats):
            self.U.append(self.U_all[ou:ou + mu[i]].view(a.shape[0], k))
            self.S.append(self.S_all[i * k:(i + 1) * k])
            self.V.append(self.V_all[ov:ov + nv[i]].view(a.shape[1], k))
            ou += mu[i]
            ov += nv[i]
        rows = []
        for a, u, s_, v in zip(mats, self.U, self.S, self.V):
            _need_cuda(a, "A")
            rows.append([a.data_ptr(), a.shape[0], a.shape[1], _rowmajor_ld(a, "A"), u.data_ptr(), k,
                         s_.data_ptr(), v.data_ptr(), k])
        self.desc = torch.tensor(rows, dtype=torch.int64, device=device)   # 9 x 8-byte fields per matrix
        self.max_m = max(a.shape[0] for a in mats)
        self.max_n = max(a.shape[1] for a in mats)
        self.status = torch.zeros(len(mats), dtype=torch.int32, device=device)


def weights_table(col_weights, device) -> torch.Tensor:
    """Device table of per-matrix weight pointers (0 for None) for rpca_batched; the
    caller keeps the weight tensors alive while the table is in use."""
    return torch.tensor([0 if w is None else w.data_ptr() for w in col_weights], dtype=torch.int64, device=device)


def rpca_batched(batch: Batch, l: int | None = None, its: int = 2, raw: bool = False, seed: int = 0,
                 col_weights=None, ws: torch.Tensor | None = None, stream=None, check: bool = True):
    """Randomized PCA of every matrix of `batch` in one launch.  col_weights: None, a
    list of per-matrix n-vectors (or None entries), or a weights_table() tensor.
    Returns (U list, S list, V list)."""
    k = batch.k
    opts = make_opts(k, l, its, raw, seed, "fp32", "cholqr")
    lib = L.load()
    count = len(batch.mats)
    need = int(lib.rpca_batched_workspace_size(count, batch.max_m, batch.max_n, C.byref(opts)))
    if need == 0:
        raise RpcaError(L.RPCA_ERR_INVALID_ARG, "rpca_batched_workspace_size")
    if ws is None or ws.numel() < need:
        ws = workspace(need, batch.desc.device)
    wptr = None
    if isinstance(col_weights, torch.Tensor):
        wptr = col_weights                    # a table from weights_table()
    elif col_weights is not None:
        wptr = weights_table(col_weights, batch.desc.device)
        batch._wkeep = (col_weights, wptr)
    code = lib.rpca_batched(count, _ptr(batch.desc), batch.max_m, batch.max_n, C.byref(opts), _ptr(wptr),
                            _ptr(batch.status), _ptr(ws), ws.numel(), _stream(stream))
    _check(code, "rpca_batched")
    if check:
        _check(rpca_read_status(ws, stream), "rpca_batched (device)")
    return batch.U, batch.S, batch.V


def rpca_batched_learned(batch: Batch, col_weights, l: int | None = None, its: int = 2, raw: bool = False,
                         seed: int = 0, resid_iters: int = 3, fallback_ratio: float = 1.1,
                         ws: torch.Tensor | None = None, est_out: torch.Tensor | None = None, stream=None,
                         check: bool = True):
    """Batched PCA with learned test-matrix weights and the per-matrix fallback to the
    plain sketch (see include/rpca.h).  batch.status afterwards: 0 kept, 1 fell back.
    Returns (U list, S list, V list, est) with est (count x 2, device): the learned
    run's residual estimate and s_{k+1} per matrix."""
    k = batch.k
    opts = make_opts(k, l, its, raw, seed, "fp32", "cholqr")
    lib = L.load()
    count = len(batch.mats)
    need = int(lib.rpca_batched_learned_workspace_size(count, batch.max_m, batch.max_n, C.byref(opts)))
    if need == 0:
        raise RpcaError(L.RPCA_ERR_INVALID_ARG, "rpca_batched_learned_workspace_size")
    if ws is None or ws.numel() < need:
        ws = workspace(need, batch.desc.device)
    if isinstance(col_weights, torch.Tensor):
        wptr = col_weights
    else:
        wptr = weights_table(col_weights, batch.desc.device)
        batch._wkeep = (col_weights, wptr)
    if est_out is None:
        est_out = torch.empty(count, 2, dtype=torch.float32, device=batch.desc.device)
    code = lib.rpca_batched_learned(count, _ptr(batch.desc), batch.max_m, batch.max_n, C.byref(opts), _ptr(wptr),
                                    int(resid_iters), float(fallback_ratio), _ptr(batch.status), _ptr(est_out),
                                    _ptr(ws), ws.numel(), _stream(stream))
    _check(code, "rpca_batched_learned")
    if check:
        _check(rpca_read_status(ws, stream), "rpca_batched_learned (device)")
    return batch.U, batch.S, batch.V, est_out


def rpca_batched_tune(batch: Batch, l: int | None = None, its: int = 2, raw: bool = False, seed: int = 0,
                      col_weights=None, ws: torch.Tensor | None = None, stream=None):
    """Time the batched kernel's pass-tile shapes on this batch and keep the fastest for later
    rpca_batched calls on batches of the same shape.  Returns ((rows_per_thread, depth),
    [ms for 2x64, 4x32, 8x32])."""
    k = batch.k
    opts = make_opts(k, l, its, raw, seed, "fp32", "cholqr")
    lib = L.load()
    count = len(batch.mats)
    need = int(lib.rpca_batched_workspace_size(count, batch.max_m, batch.max_n, C.byref(opts)))
    if need == 0:
        raise RpcaError(L.RPCA_ERR_INVALID_ARG, "rpca_batched_workspace_size")
    if ws is None or ws.numel() < need:
        ws = workspace(need, batch.desc.device)
    wptr = None
    if isinstance(col_weights, torch.Tensor):
        wptr = col_weights
    elif col_weights is not None:
        wptr = weights_table(col_weights, batch.desc.device)
        batch._wkeep = (col_weights, wptr)
    rpt = C.c_int32(0)
    depth = C.c_int32(0)
    ms = (C.c_float * 3)()
    _check(lib.rpca_batched_tune(count, _ptr(batch.desc), batch.max_m, batch.max_n, C.byref(opts), _ptr(wptr),
                                 _ptr(batch.status), _ptr(ws), ws.numel(), _stream(stream), C.byref(rpt),
                                 C.byref(depth), ms),
           "rpca_batched_tune")
    return (int(rpt.value), int(depth.value)), [float(x) for x in ms]


# ---------------------------------------------------------------------------
# learned sketch weighting
# ---------------------------------------------------------------------------
def rpca_sketch_features(A: torch.Tensor, raw: bool = False, seed: int = 0, F: torch.Tensor | None = None,
                         ws: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """The n x 16 column features of dense A (see include/rpca.h)."""
    _need_cuda(A, "A")
    lda = _rowmajor_ld(A, "A")
    m, n = A.shape
    lib = L.load()
    need = int(lib.rpca_features_workspace_size(m, n))
    if need == 0:
        raise RpcaError(L.RPCA_ERR_INVALID_ARG, "rpca_features_workspace_size")
    if ws is None or ws.numel() < need:
        ws = workspace(need, A.device)
    if F is None:
        F = torch.empty(n, L.RPCA_MLP_FEATURES, dtype=torch.float32, device=A.device)
    _check(lib.rpca_sketch_features(_ptr(A), m, n, lda, int(bool(raw)), int(seed) & ((1 << 64) - 1), _ptr(F),
                                    _ptr(ws), ws.numel(), _stream(stream)), "rpca_sketch_features")
    return F


def batch_col_offsets(batch: "Batch") -> tuple[torch.Tensor, int]:
    """(device int64 offsets of each item's first column, total columns)."""
    ns = [int(a.shape[1]) for a in batch.mats]
    offs = [0]
    for n in ns[:-1]:
        offs.append(offs[-1] + n)
    return torch.tensor(offs, dtype=torch.int64, device=batch.desc.device), sum(ns)


def rpca_batched_features(batch: "Batch", raw: bool = False, seed: int = 0, col_offsets=None,
                          F: torch.Tensor | None = None, ws: torch.Tensor | None = None,
                          stream=None) -> torch.Tensor:
    """Features of every matrix of `batch`, stacked (sum n_i) x 16 in item order."""
    if col_offsets is None:
        col_offsets, total = batch_col_offsets(batch)
    else:
        total = sum(int(a.shape[1]) for a in batch.mats)
    if F is None:
        F = torch.empty(total, L.RPCA_MLP_FEATURES, dtype=torch.float32, device=batch.desc.device)
    lib = L.load()
    need = int(lib.rpca_batched_features_workspace_size(batch.max_m))
    if ws is None or ws.numel() < need:
        ws = workspace(need, batch.desc.device)
    _check(lib.rpca_batched_features(len(batch.mats), _ptr(batch.desc), batch.max_m, int(bool(raw)),
                                     int(seed) & ((1 << 64) - 1), _ptr(col_offsets), _ptr(F), _ptr(ws),
                                     ws.numel(), _stream(stream)), "rpca_batched_features")
    return F


def rpca_mlp_pack(params: torch.Tensor, packed: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """FP32 parameters (RPCA_MLP_PARAMS) -> the packed inference blob (uint8 tensor)."""
    _need_cuda(params, "params")
    if params.numel() != L.RPCA_MLP_PARAMS or not params.is_contiguous():
        raise ValueError("params must be a contiguous vector of RPCA_MLP_PARAMS floats")
    if packed is None:
        packed = torch.empty(L.RPCA_MLP_PACKED_BYTES, dtype=torch.uint8, device=params.device)
    _check(L.load().rpca_mlp_pack(_ptr(params), _ptr(packed), _stream(stream)), "rpca_mlp_pack")
    return packed


def rpca_mlp_forward(packed: torch.Tensor, F: torch.Tensor, want_y: bool = True, want_d: bool = True,
                     ws: torch.Tensor | None = None, stream=None, check: bool = True, y=None, d=None):
    """(y, d) for the rows of F (N x 16) on the tensor cores; either may be None.
    y / d: optional preallocated outputs (N floats each)."""
    _need_cuda(F, "F")
    if F.dim() != 2 or F.shape[1] != L.RPCA_MLP_FEATURES or not F.is_contiguous():
        raise ValueError("F must be a contiguous N x 16 tensor")
    N = F.shape[0]
    if y is None and want_y:
        y = torch.empty(N, dtype=torch.float32, device=F.device)
    if d is None and want_d:
        d = torch.empty(N, dtype=torch.float32, device=F.device)
    lib = L.load()
    if ws is None:
        ws = workspace(int(lib.rpca_mlp_forward_workspace_size()), F.device)
    _check(lib.rpca_mlp_forward(_ptr(packed), _ptr(F), N, _ptr(y), _ptr(d), _ptr(ws), ws.numel(),
                                _stream(stream)), "rpca_mlp_forward")
    if check:
        _check(rpca_read_status(ws, stream), "rpca_mlp_forward (device)")
    return y, d


def rpca_mlp_loss_grad(params: torch.Tensor, F: torch.Tensor, t: torch.Tensor, grad: torch.Tensor | None = None,
                       loss: torch.Tensor | None = None, ws: torch.Tensor | None = None, stream=None):
    """(loss tensor [1], grad tensor [RPCA_MLP_PARAMS]) of the mean squared error."""
    for x, nm in ((params, "params"), (F, "F"), (t, "t")):
        _need_cuda(x, nm)
        if not x.is_contiguous():
            raise ValueError(f"{nm} must be contiguous")
    N = F.shape[0]
    lib = L.load()
    need = int(lib.rpca_mlp_grad_workspace_size(N))
    if ws is None or ws.numel() < need:
        ws = workspace(need, F.device)
    if grad is None:
        grad = torch.empty(L.RPCA_MLP_PARAMS, dtype=torch.float32, device=F.device)
    if loss is None:
        loss = torch.empty(1, dtype=torch.float32, device=F.device)
    _check(lib.rpca_mlp_loss_grad(_ptr(params), _ptr(F), _ptr(t), N, _ptr(grad), _ptr(loss), _ptr(ws), ws.numel(),
                                  _stream(stream)), "rpca_mlp_loss_grad")
    return loss, grad


def rpca_mlp_adam(params, grad, m1, m2, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
                  eps: float = 1e-8, stream=None) -> None:
    _check(L.load().rpca_mlp_adam(_ptr(params), _ptr(grad), _ptr(m1), _ptr(m2), int(step), float(lr), float(beta1),
                                  float(beta2), float(eps), _stream(stream)), "rpca_mlp_adam")


def rpca_leverage_target(V: torch.Tensor, k: int, t: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    _need_cuda(V, "V")
    ldv = _rowmajor_ld(V, "V")
    n = V.shape[0]
    if t is None:
        t = torch.empty(n, dtype=torch.float32, device=V.device)
    _check(L.load().rpca_leverage_target(_ptr(V), n, ldv, int(k), _ptr(t), _stream(stream)), "rpca_leverage_target")
    return t


def rpca_dense_learned(A: torch.Tensor, packed: torch.Tensor, k: int, l: int | None = None, its: int = 2,
                       raw: bool = False, seed: int = 0, precision: str = "fp32", resid_iters: int = 8,
                       fallback_ratio: float = 1.1, ws: torch.Tensor | None = None, stream=None):
    """Learned-sketch PCA with fallback.  Returns (U, S, V, info) with info =
    {"fell_back": bool, "est": residual estimate of the learned run, "s_k1": s_{k+1}}."""
    _need_cuda(A, "A")
    lda = _rowmajor_ld(A, "A")
    m, n = A.shape
    opts = make_opts(k, l, its, raw, seed, precision, "cholqr")
    lib = L.load()
    need = int(lib.rpca_dense_learned_workspace_size(m, n, C.byref(opts)))
    if need == 0:
        raise RpcaError(L.RPCA_ERR_INVALID_ARG, "rpca_dense_learned_workspace_size")
    if ws is None or ws.numel() < need:
        ws = workspace(need, A.device)
    U = torch.empty(m, k, dtype=torch.float32, device=A.device)
    S = torch.empty(k, dtype=torch.float32, device=A.device)
    V = torch.empty(n, k, dtype=torch.float32, device=A.device)
    est = (C.c_double * 2)()
    code = lib.rpca_dense_learned(_ptr(A), m, n, lda, C.byref(opts), _ptr(packed), int(resid_iters),
                                  float(fallback_ratio), _ptr(U), k, _ptr(S), _ptr(V), k, est, _ptr(ws), ws.numel(),
                                  _stream(stream))
    _check(code, "rpca_dense_learned")
    return U, S, V, {"fell_back": code == L.RPCA_FELL_BACK, "est": est[0], "s_k1": est[1]}

// rpca_dense_pass_noalloc: one product of the method with its scratch held in
// a fixed buffer that is part of the library image, for callers that may not
// allocate device memory.
//
// Who cannot allocate: code running inside a host framework that owns all
// device memory through its own pool or caching allocator and hands out only
// buffers it sized itself; code on a latency-critical path where cudaMalloc's
// implicit device synchronisation (or a failure under memory pressure) is not
// acceptable; code that must not grow the process's device footprint once it
// has started.  Such a caller still passes A, B and C; everything else the
// product needs (status word, split-K partials, split BF16 block operand) comes
// from g_pass_scratch below.
#include "internal.cuh"

// One buffer per device, created when the library's device code is loaded on
// that device and held until the process exits.
static __device__ __align__(256) unsigned char g_pass_scratch[RPCA_NOALLOC_SCRATCH_BYTES];

namespace {

// Device address of g_pass_scratch on the current device.  Host code cannot
// use the symbol itself (on the host it names a stand-in, not device memory).
// The address is looked up on every call rather than cached: the lookup is a
// host-side table query, and a cached address would go stale if the caller's
// framework reset the device's primary context (the module, and with it the
// buffer, is then loaded again at another address).
int scratch_address(void **out) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_pass_scratch) != cudaSuccess || !p) return RPCA_ERR_CUDA;
    *out = p;
    return RPCA_OK;
}

}  // namespace

extern "C" int rpca_dense_pass_noalloc(const float *A, int64_t m, int64_t n, int64_t lda, int32_t adjoint,
                                       const float *B, int32_t w, float *C, int32_t precision,
                                       rpca_stream_t stream) {
    if (!A || !B || !C || m < 1 || n < 1 || lda < n || w < 8 || w > 256 || w % 8) return RPCA_ERR_INVALID_ARG;
    if (precision != RPCA_PREC_FP32 && precision != RPCA_PREC_BF16X3) return RPCA_ERR_INVALID_ARG;
    const size_t need = rpca_dense_pass_workspace_size(m, n, w, adjoint, precision);
    if (need == 0) return RPCA_ERR_INVALID_ARG;
    if (need > (size_t)RPCA_NOALLOC_SCRATCH_BYTES) return RPCA_ERR_WORKSPACE;   // too large for the fixed buffer
    void *ws = nullptr;
    RPCA_TRY(scratch_address(&ws));
    // rpca_dense_pass clears the status word on `stream` before its kernels run;
    // the partials and the split operand are fully overwritten by each call.
    return rpca_dense_pass(A, m, n, lda, adjoint, B, w, C, precision, ws, (size_t)RPCA_NOALLOC_SCRATCH_BYTES,
                           stream);
}

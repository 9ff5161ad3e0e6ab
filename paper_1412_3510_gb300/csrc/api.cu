// Small C-ABI helpers: defaults, status words and strings, launch accounting.
#include "internal.cuh"

#include <atomic>

namespace rpca {

static std::atomic<int64_t> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

int check_launch() {
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? RPCA_OK : RPCA_ERR_CUDA;
}

int num_sms() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 148;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
        return 148;
    return n;
}

}  // namespace rpca

extern "C" void rpca_default_opts(rpca_opts *o, int32_t k) {
    if (!o) return;
    o->k = k;
    o->l = k + 2;            // Section 7: l = k + 2 is the default oversampling
    o->its = 2;              // Section 5/7: its = 2 is the default
    o->raw = 0;              // PCA centres the columns (Section 2)
    o->seed = 0;
    o->precision = RPCA_PREC_FP32;
    o->renorm = RPCA_RENORM_CHOLQR;
    o->omega = nullptr;
    o->col_weights = nullptr;
}

extern "C" int rpca_read_status(const void *ws, rpca_stream_t stream, int32_t *status) {
    if (!ws || !status) return RPCA_ERR_INVALID_ARG;
    rpca::DevStatus h;
    if (cudaMemcpyAsync(&h, ws, sizeof(h), cudaMemcpyDeviceToHost, (cudaStream_t)stream) != cudaSuccess)
        return RPCA_ERR_CUDA;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return RPCA_ERR_CUDA;
    if (h.status < 0) *status = h.status;
    else *status = (h.flags & 1) ? RPCA_FELL_BACK : RPCA_OK;
    return RPCA_OK;
}

extern "C" const char *rpca_status_string(int status) {
    switch (status) {
        case RPCA_OK: return "ok";
        case RPCA_FELL_BACK: return "ok (fell back)";
        case RPCA_ERR_INVALID_ARG: return "invalid argument";
        case RPCA_ERR_WORKSPACE: return "workspace missing, too small or misaligned";
        case RPCA_ERR_CUDA: return "CUDA launch or runtime error";
        case RPCA_ERR_NONFINITE: return "non-finite values reached a factorisation";
        case RPCA_ERR_BREAKDOWN: return "factorisation broke down after its fallback";
        case RPCA_ERR_TIMEOUT: return "a bounded device wait expired";
        case RPCA_ERR_UNSUPPORTED: return "option combination not supported";
        default: return "unknown status";
    }
}

extern "C" int64_t rpca_launch_count(void) { return rpca::g_launches.load(); }

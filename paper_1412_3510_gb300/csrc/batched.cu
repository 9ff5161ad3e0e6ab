// Batched randomized PCA: many small, uneven dense matrices in one launch.
//
// The method is the same as rpca_dense (Sections 2 and 5: Gaussian sketch,
// power iterations renormalised after every product, final orthonormal basis,
// B = Q^* A_c, SVD of the small factor, U = Q W).  For thousands of matrices of
// a few MB each, per-matrix launches would dominate, so one persistent kernel
// runs whole PCAs: each CTA takes the next matrix from a work queue (largest
// first) and carries it through every step with block-wide barriers only --
// no CTA ever waits on another, so there are no cross-CTA spin waits.
//
// Per CTA: the n-side block (Omega, X, B^*) lives in shared memory (n * lp <=
// kMaxNL floats); the m-side block Y lives in a per-CTA slot of the workspace
// (L2-resident for these sizes); the l x l Cholesky factors and the Jacobi SVD
// (l <= 32) are done by warps in shared memory.  Products stream A through
// shared-memory tiles with FP32 FFMA.
#include "batched_kernels.cuh"

#include <map>
#include <mutex>
#include <tuple>

namespace rpca {

namespace {

// Work order: descending m * n (ties by index), by rank counting with the sizes staged
// through shared memory 2048 at a time.
__global__ void __launch_bounds__(256) order_kernel(const Item *__restrict__ items, int count, int32_t *__restrict__ order) {
    __shared__ int64_t w[2048];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t wi = i < count ? items[i].m * items[i].n : 0;
    int rank = 0;
    for (int j0 = 0; j0 < count; j0 += 2048) {
        __syncthreads();
        for (int j = threadIdx.x; j < 2048 && j0 + j < count; j += blockDim.x) w[j] = items[j0 + j].m * items[j0 + j].n;
        __syncthreads();
        const int jn = min(2048, count - j0);
        for (int j = 0; j < jn; ++j) rank += (w[j] > wi) || (w[j] == wi && j0 + j < i);
    }
    if (i < count) order[rank] = i;
}

__global__ void check_items_kernel(const Item *__restrict__ items, int count, int l, int k, int64_t max_m,
                                   int32_t *__restrict__ item_status, const int32_t *__restrict__ active,
                                   int *__restrict__ queue, DevStatus *st) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *queue = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        if (active && active[i] == 0) continue;                            // skipped: status untouched
        const bool ok = item_ok(items[i], l, k, max_m);
        if (item_status) item_status[i] = ok ? 1 : RPCA_ERR_INVALID_ARG;     // 1: pending
        if (!ok) dev_fail(st, RPCA_ERR_INVALID_ARG);
    }
}

}  // namespace

}  // namespace rpca

namespace {

struct BatchLayout {
    size_t status = 0, queue = 0, order = 0, slots = 0, total = 0;
    int64_t slot_floats = 0;
};

BatchLayout batch_layout(int32_t count, int64_t max_m, int l) {
    BatchLayout B;
    size_t off = 0;
    auto take = [&](size_t b) { const size_t o = off; off = (off + b + 255) & ~(size_t)255; return o; };
    const int lp = (int)rpca::round_up(l + 1, 8);
    B.status = take(sizeof(rpca::DevStatus));
    B.queue = take(256);
    B.order = take((size_t)count * 4);
    B.slot_floats = rpca::round_up(max_m * lp, 64);
    B.slots = take((size_t)rpca::num_sms() * B.slot_floats * 4);
    B.total = off;
    return B;
}

}  // namespace

extern "C" size_t rpca_batched_workspace_size(int32_t count, int64_t max_m, int64_t max_n, const rpca_opts *o) {
    if (!o || count < 0 || max_m < 1 || max_n < 1 || o->l < 1 || o->l > 32 || o->k < 1 || o->k > o->l) return 0;
    return batch_layout(count, max_m, o->l).total;
}

namespace {

// Tuned pass-tile shapes (index into kShapes), keyed by the batch's shape and the
// method's parameters; filled by rpca_batched_tune.
using TuneKey = std::tuple<int32_t, int64_t, int64_t, int32_t, int32_t, int32_t, int32_t>;
std::mutex g_tune_mutex;
std::map<TuneKey, int> g_tuned;
struct Shape { int rows, depth; };
constexpr int kNumShapes = 3;
constexpr Shape kShapes[kNumShapes] = {{2, 64}, {4, 32}, {8, 32}};
constexpr int kDefaultShape = 1;             // 4 rows, 32 deep

TuneKey tune_key(int32_t count, int64_t max_m, int64_t max_n, const rpca_opts *o) {
    return TuneKey(count, max_m, max_n, o->l, o->k, o->its, o->raw ? 1 : 0);
}

int tuned_rpt(const TuneKey &key) {
    std::lock_guard<std::mutex> g(g_tune_mutex);
    const auto it = g_tuned.find(key);
    return it == g_tuned.end() ? kDefaultShape : it->second;
}

int check_args(int32_t count, const rpca_mat_desc *descs, int64_t max_m, int64_t max_n, const rpca_opts *o,
               const void *ws, size_t ws_bytes) {
    if (!o || count < 0 || (count > 0 && !descs) || o->l < 1 || o->l > 32 || o->k < 1 || o->k > o->l || o->its < 0 ||
        o->its > 1000 || max_m < 1 || max_n < 1 || count > 65536)
        return RPCA_ERR_INVALID_ARG;
    if (o->omega || o->renorm != RPCA_RENORM_CHOLQR || rpca::small_fp64(o->precision)) return RPCA_ERR_UNSUPPORTED;
    const size_t need = rpca_batched_workspace_size(count, max_m, max_n, o);
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0 || ws_bytes < need) return RPCA_ERR_WORKSPACE;
    return RPCA_OK;
}

}  // namespace

namespace rpca {

int run_batched(int32_t count, const rpca_mat_desc *descs, int64_t max_m, const rpca_opts *o,
                const float *const *col_weights, int32_t *item_status, void *ws, cudaStream_t s, int shape,
                const int32_t *active, float *sk1) {
    static_assert(sizeof(rpca_mat_desc) == sizeof(rpca::Item), "descriptor layout");
    const BatchLayout B = batch_layout(count, max_m, o->l);
    char *base = reinterpret_cast<char *>(ws);
    auto *st = reinterpret_cast<rpca::DevStatus *>(base + B.status);
    auto *queue = reinterpret_cast<int *>(base + B.queue);
    auto *order = reinterpret_cast<int32_t *>(base + B.order);
    auto *items = reinterpret_cast<const rpca::Item *>(descs);
    if (cudaMemsetAsync(st, 0, sizeof(rpca::DevStatus), s) != cudaSuccess) return RPCA_ERR_CUDA;
    rpca::check_items_kernel<<<(int)rpca::cdiv(count, 256), 256, 0, s>>>(items, count, o->l, o->k, max_m, item_status,
                                                                         active, queue, st);
    RPCA_CHECK_LAUNCH();
    rpca::order_kernel<<<(int)rpca::cdiv(count, 256), 256, 0, s>>>(items, count, order);
    RPCA_CHECK_LAUNCH();
    rpca::BatchLaunch a{items, order, count, o->l, o->k, o->its, o->raw, o->seed, col_weights, item_status, active,
                        sk1, queue, reinterpret_cast<float *>(base + B.slots), B.slot_floats, max_m, rpca::num_sms(),
                        s};
    switch (shape) {
        case 0: return rpca::launch_batched_r2k64(a);
        case 2: return rpca::launch_batched_r8k32(a);
        default: return rpca::launch_batched_r4k32(a);
    }
}

int batched_shape(int32_t count, int64_t max_m, int64_t max_n, const rpca_opts *o) {
    return tuned_rpt(tune_key(count, max_m, max_n, o));
}

int check_batched_args(int32_t count, const rpca_mat_desc *descs, int64_t max_m, int64_t max_n, const rpca_opts *o,
                       const void *ws, size_t ws_bytes) {
    return check_args(count, descs, max_m, max_n, o, ws, ws_bytes);
}

}  // namespace rpca

extern "C" int rpca_batched(int32_t count, const rpca_mat_desc *descs, int64_t max_m, int64_t max_n,
                            const rpca_opts *o, const float *const *col_weights, int32_t *item_status, void *ws,
                            size_t ws_bytes, rpca_stream_t stream) {
    RPCA_TRY(check_args(count, descs, max_m, max_n, o, ws, ws_bytes));
    if (count == 0) return RPCA_OK;
    return rpca::run_batched(count, descs, max_m, o, col_weights, item_status, ws, (cudaStream_t)stream,
                             tuned_rpt(tune_key(count, max_m, max_n, o)), nullptr, nullptr);
}

extern "C" int rpca_batched_tune(int32_t count, const rpca_mat_desc *descs, int64_t max_m, int64_t max_n,
                                 const rpca_opts *o, const float *const *col_weights, int32_t *item_status, void *ws,
                                 size_t ws_bytes, rpca_stream_t stream, int32_t *rows_per_thread, int32_t *depth,
                                 float *ms) {
    RPCA_TRY(check_args(count, descs, max_m, max_n, o, ws, ws_bytes));
    if (count == 0) return RPCA_OK;
    cudaStream_t s = (cudaStream_t)stream;
    float best_ms = 0.f;
    int best = kDefaultShape;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return RPCA_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return RPCA_ERR_CUDA; }
    int rc = RPCA_OK;
    for (int c = 0; c < kNumShapes && rc == RPCA_OK; ++c) {
        rc = rpca::run_batched(count, descs, max_m, o, col_weights, item_status, ws, s, c, nullptr, nullptr);  // warm-up
        if (rc != RPCA_OK) break;
        if (cudaEventRecord(e0, s) != cudaSuccess) { rc = RPCA_ERR_CUDA; break; }
        rc = rpca::run_batched(count, descs, max_m, o, col_weights, item_status, ws, s, c, nullptr, nullptr);
        if (rc != RPCA_OK) break;
        float t = 0.f;
        if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
            rc = RPCA_ERR_CUDA;
            break;
        }
        if (ms) ms[c] = t;
        if (c == 0 || t < best_ms) { best_ms = t; best = c; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != RPCA_OK) return rc;
    {
        std::lock_guard<std::mutex> g(g_tune_mutex);
        g_tuned[tune_key(count, max_m, max_n, o)] = best;
    }
    if (rows_per_thread) *rows_per_thread = kShapes[best].rows;
    if (depth) *depth = kShapes[best].depth;
    return RPCA_OK;
}

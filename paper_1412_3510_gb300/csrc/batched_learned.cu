// The batched form with the learned test-matrix weighting and its fallback.
//
// rpca_batched runs every matrix with its weighted test matrix diag(d) Omega.  Each
// matrix's residual ||A_c - U S V^T|| is then estimated by the power method of
// Section 4 (a few iterations from the random start the dense estimator uses), and
// compared with fallback_ratio * s_{k+1}, s_{k+1} the (k+1)-th singular value of the
// same run's rank-l approximation.  The matrices that miss it are run again with the
// plain Gaussian test matrix, in one more launch of the batched kernel that skips
// every other matrix; their status becomes RPCA_FELL_BACK.
#include "batched_kernels.cuh"

namespace rpca {

int run_batched(int32_t count, const rpca_mat_desc *descs, int64_t max_m, const rpca_opts *o,
                const float *const *col_weights, int32_t *item_status, void *ws, cudaStream_t s, int shape,
                const int32_t *active, float *sk1);
int batched_shape(int32_t count, int64_t max_m, int64_t max_n, const rpca_opts *o);
int check_batched_args(int32_t count, const rpca_mat_desc *descs, int64_t max_m, int64_t max_n, const rpca_opts *o,
                       const void *ws, size_t ws_bytes);

namespace {

constexpr int kResidThreads = 512;

__device__ float block_sum(float v, float *red) {
#pragma unroll
    for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    float t = 0.f;
    if (threadIdx.x < 32) {
        t = threadIdx.x < (int)(blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
#pragma unroll
        for (int off = 16; off; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
        if (threadIdx.x == 0) red[32] = t;
    }
    __syncthreads();
    return red[32];
}

// Section 4's power method on E = A_c - U diag(S) V^T, one CTA per matrix: x0 from the
// Philox stream (seed, 1) normalised; each iteration y = A_c x - U (S .* (V^T x)),
// z = A_c^T y - V (S .* (U^T y)), lambda = |z|, x = z / lambda; est = sqrt(lambda).
// A_c x is A x minus its row mean, A_c^T y is A^T (y minus its mean).  Only items with
// status 0 (computed) are estimated; the others get est = -1.
__global__ void __launch_bounds__(kResidThreads)
batched_resid_kernel(const Item *__restrict__ items, int count, int k, int raw, int iters, uint64_t seed,
                     const int32_t *__restrict__ status, float *__restrict__ est) {
    extern __shared__ float sm[];
    __shared__ float red[33];
    __shared__ float tk[32], uk[32];
    const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, lane = tid & 31, nwarps = nt >> 5;
    for (int idx = blockIdx.x; idx < count; idx += gridDim.x) {
        if (status && status[idx] != 0) {
            if (tid == 0) est[idx] = -1.f;
            continue;
        }
        const Item it = items[idx];
        const int64_t m = it.m, n = it.n;
        float *x = sm, *y = sm + n;
        for (int64_t j = tid; j < n; j += nt) {
            float z[4];
            gauss4((uint64_t)(j >> 2), seed, 1, z);
            x[j] = z[j & 3];
        }
        __syncthreads();
        float s2 = 0.f;
        for (int64_t j = tid; j < n; j += nt) s2 = fmaf(x[j], x[j], s2);
        float nrm = sqrtf(block_sum(s2, red));
        for (int64_t j = tid; j < n; j += nt) x[j] /= nrm;
        __syncthreads();
        float lambda = 0.f;
        for (int q = 0; q < iters; ++q) {
            // t = S .* (V^T x)
            for (int r = warp; r < k; r += nwarps) {
                float v = 0.f;
                for (int64_t j = lane; j < n; j += 32) v = fmaf(it.V[j * it.ldv + r], x[j], v);
#pragma unroll
                for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
                if (lane == 0) tk[r] = v * it.S[r];
            }
            // y = A x (a warp per row)
            for (int64_t i = warp; i < m; i += nwarps) {
                const float *a = it.A + i * it.lda;
                float v = 0.f;
                for (int64_t j = lane; j < n; j += 32) v = fmaf(a[j], x[j], v);
#pragma unroll
                for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
                if (lane == 0) y[i] = v;
            }
            __syncthreads();
            float mean = 0.f;
            if (!raw) {
                float sy = 0.f;
                for (int64_t i = tid; i < m; i += nt) sy += y[i];
                mean = block_sum(sy, red) / (float)m;
            }
            for (int64_t i = tid; i < m; i += nt) {
                float v = y[i] - mean;
                for (int r = 0; r < k; ++r) v = fmaf(-it.U[i * it.ldu + r], tk[r], v);
                y[i] = v;
            }
            __syncthreads();
            // u = S .* (U^T y); y centred for A_c^T
            for (int r = warp; r < k; r += nwarps) {
                float v = 0.f;
                for (int64_t i = lane; i < m; i += 32) v = fmaf(it.U[i * it.ldu + r], y[i], v);
#pragma unroll
                for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
                if (lane == 0) uk[r] = v * it.S[r];
            }
            if (!raw) {
                float sy = 0.f;
                for (int64_t i = tid; i < m; i += nt) sy += y[i];
                const float my = block_sum(sy, red) / (float)m;
                for (int64_t i = tid; i < m; i += nt) y[i] -= my;
            }
            __syncthreads();
            // x = A^T y - V u (a thread per column, rows streamed)
            float s2z = 0.f;
            for (int64_t j = tid; j < n; j += nt) {
                float v0 = 0.f, v1 = 0.f, v2 = 0.f, v3 = 0.f;         // independent chains
                int64_t i = 0;
                for (; i + 4 <= m; i += 4) {
                    v0 = fmaf(it.A[i * it.lda + j], y[i], v0);
                    v1 = fmaf(it.A[(i + 1) * it.lda + j], y[i + 1], v1);
                    v2 = fmaf(it.A[(i + 2) * it.lda + j], y[i + 2], v2);
                    v3 = fmaf(it.A[(i + 3) * it.lda + j], y[i + 3], v3);
                }
                for (; i < m; ++i) v0 = fmaf(it.A[i * it.lda + j], y[i], v0);
                float v = (v0 + v1) + (v2 + v3);
                for (int r = 0; r < k; ++r) v = fmaf(-it.V[j * it.ldv + r], uk[r], v);
                x[j] = v;
                s2z = fmaf(v, v, s2z);
            }
            lambda = sqrtf(block_sum(s2z, red));
            if (lambda == 0.f) break;
            for (int64_t j = tid; j < n; j += nt) x[j] /= lambda;
            __syncthreads();
        }
        if (tid == 0) est[idx] = sqrtf(lambda);
        __syncthreads();
    }
}

// Per item: fall back when the learned run's estimate exceeds ratio * s_{k+1} (l > k).
__global__ void fallback_flags_kernel(int count, int l, int k, float ratio, const int32_t *__restrict__ status,
                                      const float *__restrict__ est, const float *__restrict__ sk1,
                                      int32_t *__restrict__ redo) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
        redo[i] = (l > k && status[i] == 0 && est[i] > ratio * sk1[i]) ? 1 : 0;
}

// item_status[i] = RPCA_FELL_BACK for a redone item that the plain run computed, its own
// status otherwise; est_out (optional): the learned run's estimate and s_{k+1}.
__global__ void fallback_merge_kernel(int count, const int32_t *__restrict__ redo, const int32_t *__restrict__ st1,
                                      const int32_t *__restrict__ st2, const float *__restrict__ est,
                                      const float *__restrict__ sk1, int32_t *__restrict__ item_status,
                                      float *__restrict__ est_out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        if (item_status) item_status[i] = redo[i] ? (st2[i] == 0 ? RPCA_FELL_BACK : st2[i]) : st1[i];
        if (est_out) {
            est_out[2 * i] = est[i];
            est_out[2 * i + 1] = sk1[i];
        }
    }
}

struct LearnedLayout {
    size_t batched = 0, st1 = 0, st2 = 0, est = 0, sk1 = 0, redo = 0, total = 0;
};

LearnedLayout learned_layout(int32_t count, size_t batched_bytes) {
    LearnedLayout Lw;
    size_t off = 0;
    auto take = [&](size_t b) { const size_t o = off; off = (off + b + 255) & ~(size_t)255; return o; };
    Lw.batched = take(batched_bytes);
    Lw.st1 = take((size_t)count * 4);
    Lw.st2 = take((size_t)count * 4);
    Lw.est = take((size_t)count * 4);
    Lw.sk1 = take((size_t)count * 4);
    Lw.redo = take((size_t)count * 4);
    Lw.total = off;
    return Lw;
}

}  // namespace
}  // namespace rpca

extern "C" size_t rpca_batched_learned_workspace_size(int32_t count, int64_t max_m, int64_t max_n,
                                                      const rpca_opts *o) {
    const size_t b = rpca_batched_workspace_size(count, max_m, max_n, o);
    if (b == 0) return 0;
    return rpca::learned_layout(count, b).total;
}

extern "C" int rpca_batched_learned(int32_t count, const rpca_mat_desc *descs, int64_t max_m, int64_t max_n,
                                    const rpca_opts *o, const float *const *col_weights, int32_t resid_iters,
                                    float fallback_ratio, int32_t *item_status, float *est_out, void *ws,
                                    size_t ws_bytes, rpca_stream_t stream) {
    if (!o || resid_iters < 1 || resid_iters > 1000 || !(fallback_ratio > 0.f)) return RPCA_ERR_INVALID_ARG;
    const size_t bbytes = rpca_batched_workspace_size(count, max_m, max_n, o);
    RPCA_TRY(rpca::check_batched_args(count, descs, max_m, max_n, o, ws, bbytes));
    const rpca::LearnedLayout Lw = rpca::learned_layout(count, bbytes);
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0 || ws_bytes < Lw.total) return RPCA_ERR_WORKSPACE;
    if (count == 0) return RPCA_OK;
    cudaStream_t s = (cudaStream_t)stream;
    char *b = reinterpret_cast<char *>(ws);
    auto *st1 = reinterpret_cast<int32_t *>(b + Lw.st1);
    auto *st2 = reinterpret_cast<int32_t *>(b + Lw.st2);
    auto *est = reinterpret_cast<float *>(b + Lw.est);
    auto *sk1 = reinterpret_cast<float *>(b + Lw.sk1);
    auto *redo = reinterpret_cast<int32_t *>(b + Lw.redo);
    const int shape = rpca::batched_shape(count, max_m, max_n, o);
    // 1. the learned test matrix
    RPCA_TRY(rpca::run_batched(count, descs, max_m, o, col_weights, st1, b + Lw.batched, s, shape, nullptr, sk1));
    // 2. Section 4's estimate per matrix
    const size_t smem = (size_t)(max_m + max_n) * sizeof(float);
    if (cudaFuncSetAttribute(rpca::batched_resid_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return RPCA_ERR_CUDA;
    const int grid = (int)std::min<int64_t>(count, (int64_t)rpca::num_sms() * 2);
    rpca::batched_resid_kernel<<<grid, rpca::kResidThreads, smem, s>>>(
        reinterpret_cast<const rpca::Item *>(descs), count, o->k, o->raw, resid_iters, o->seed, st1, est);
    RPCA_CHECK_LAUNCH();
    const int g2 = (int)rpca::cdiv(count, 256);
    rpca::fallback_flags_kernel<<<g2, 256, 0, s>>>(count, o->l, o->k, fallback_ratio, st1, est, sk1, redo);
    RPCA_CHECK_LAUNCH();
    // 3. the plain test matrix for the matrices that missed
    if (cudaMemsetAsync(st2, 0, (size_t)count * 4, s) != cudaSuccess) return RPCA_ERR_CUDA;
    RPCA_TRY(rpca::run_batched(count, descs, max_m, o, nullptr, st2, b + Lw.batched, s, shape, redo, nullptr));
    rpca::fallback_merge_kernel<<<g2, 256, 0, s>>>(count, redo, st1, st2, est, sk1, item_status, est_out);
    RPCA_CHECK_LAUNCH();
    return RPCA_OK;
}

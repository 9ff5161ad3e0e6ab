// Column features for the learned weighting of the test matrix.
//
// One pass over A gathers, per column j: the shifted sums of a_ij - a_0j and
// of its square (centring without cancellation for columns that are nearly
// constant), the column's max and min, and the coarse sketch
// S[r, j] = sum_i G[i, r] (a_ij - a_0j) with G an m x 8 N(0,1) matrix from the
// Philox stream (seed, 2).  Finishing the column (centred on c_j unless raw):
//   q_j = sum_i (a_ij - c_j)^2, x_j = max_i |a_ij - c_j|,
//   S[r, j] -= (sum_i G[i, r]) (c_j - a_0j)
// and, with qbar = mean q, tau = 1e-12 qbar + 1e-30, rho_r = rms_j S[r, j],
// the 16 features of column j are
//   log((q_j + tau) / (qbar + tau)), c_j / sqrt(qbar / m + tau),
//   log((x_j^2 m + tau) / (q_j + tau)) / 4, S[0..7, j] / (rho_r + 1e-30),
//   log(m) / 8, log(n) / 8, 0, 0, 0.
// Dense A: a multi-CTA pass (column strips x row splits) and three small
// finishing kernels.  Batched: one CTA per matrix, every item reading the rows
// of one G drawn for the largest m (G's rows do not depend on m).
#include "internal.cuh"

namespace rpca {

namespace {

constexpr int kStrip = 128;           // columns per CTA strip (32 lanes x 4)
constexpr int kThreads = 256;
constexpr int kQ = 12;                // s1, s2, max, min, S[8]
constexpr int kSk = 8;                // sketch rows
constexpr int kWarps = kThreads / 32;

struct ColStats {
    float c, q, x, S[kSk];
};

// Finish one column from its shifted sums (see the file comment).
__device__ __forceinline__ ColStats finish_column(float shift, float s1, float s2, float mx, float mn,
                                                  const float *Sd, const float *gsum, int64_t m, int raw) {
    ColStats cs;
    const float fm = (float)m;
    cs.c = raw ? 0.f : shift + s1 / fm;
    cs.q = raw ? s2 : fmaxf(s2 - s1 * (s1 / fm), 0.f);
    cs.x = fmaxf(mx - cs.c, cs.c - mn);
    const float dc = cs.c - shift;
#pragma unroll
    for (int r = 0; r < kSk; ++r) cs.S[r] = Sd[r] - gsum[r] * dc;
    return cs;
}

__device__ __forceinline__ void write_features(float *Fj, const ColStats &cs, float qbar, const float *rho,
                                               int64_t m, int64_t n) {
    const float tau = 1e-12f * qbar + 1e-30f;
    const float fm = (float)m;
    Fj[0] = logf((cs.q + tau) / (qbar + tau));
    Fj[1] = cs.c / sqrtf(qbar / fm + tau);
    Fj[2] = 0.25f * logf((cs.x * cs.x * fm + tau) / (cs.q + tau));
#pragma unroll
    for (int r = 0; r < kSk; ++r) Fj[3 + r] = cs.S[r] / (rho[r] + 1e-30f);
    Fj[11] = logf(fm) * 0.125f;
    Fj[12] = logf((float)n) * 0.125f;
    Fj[13] = 0.f;
    Fj[14] = 0.f;
    Fj[15] = 0.f;
}

// ---------------------------------------------------------------------------
// one 128-column strip over rows [r0, r1): lanes own 4 adjacent columns, the 8
// warps take interleaved rows, 4 rows in flight per warp; per-warp partials to red
// (kWarps x kQ x kStrip)
// ---------------------------------------------------------------------------
template <bool VEC>
__device__ __forceinline__ void strip_pass(const float *__restrict__ A, int64_t n, int64_t lda, int raw,
                                           const float *__restrict__ G, int64_t cb, int64_t r0, int64_t r1,
                                           float *red) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t col0 = cb + 4 * lane;
    bool live[4];
    float shift[4], s1[4], s2[4], mx[4], mn[4], Sd[4][kSk];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        live[q] = col0 + q < n;
        shift[q] = (!raw && live[q]) ? A[col0 + q] : 0.f;
        s1[q] = s2[q] = 0.f;
        mx[q] = -INFINITY;
        mn[q] = INFINITY;
#pragma unroll
        for (int r = 0; r < kSk; ++r) Sd[q][r] = 0.f;
    }
    constexpr int kU = 4;                        // rows in flight per warp
    for (int64_t i0 = r0 + warp; i0 < r1; i0 += kWarps * kU) {
        float a[kU][4], g[kU][kSk];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int64_t i = i0 + (int64_t)u * kWarps;
            if (i < r1) {
                const float4 g0 = __ldg(reinterpret_cast<const float4 *>(G + i * kSk));
                const float4 g1 = __ldg(reinterpret_cast<const float4 *>(G + i * kSk) + 1);
                g[u][0] = g0.x; g[u][1] = g0.y; g[u][2] = g0.z; g[u][3] = g0.w;
                g[u][4] = g1.x; g[u][5] = g1.y; g[u][6] = g1.z; g[u][7] = g1.w;
                const float *row = A + i * lda + col0;
                if (VEC && live[3]) {
                    const float4 v = __ldg(reinterpret_cast<const float4 *>(row));
                    a[u][0] = v.x; a[u][1] = v.y; a[u][2] = v.z; a[u][3] = v.w;
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q) a[u][q] = live[q] ? __ldg(row + q) : 0.f;
                }
            } else {
#pragma unroll
                for (int r = 0; r < kSk; ++r) g[u][r] = 0.f;
#pragma unroll
                for (int q = 0; q < 4; ++q) a[u][q] = 0.f;
            }
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            if (i0 + (int64_t)u * kWarps >= r1) break;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float d = a[u][q] - shift[q];
                s1[q] += d;
                s2[q] = fmaf(d, d, s2[q]);
                mx[q] = fmaxf(mx[q], a[u][q]);
                mn[q] = fminf(mn[q], a[u][q]);
#pragma unroll
                for (int r = 0; r < kSk; ++r) Sd[q][r] = fmaf(g[u][r], d, Sd[q][r]);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        float *o = red + (warp * kQ) * kStrip + 4 * lane + q;
        o[0 * kStrip] = s1[q];
        o[1 * kStrip] = s2[q];
        o[2 * kStrip] = mx[q];
        o[3 * kStrip] = mn[q];
#pragma unroll
        for (int r = 0; r < kSk; ++r) o[(4 + r) * kStrip] = Sd[q][r];
    }
}

// quantity qty of strip column c, combined over the warps in a fixed order
__device__ __forceinline__ float strip_combine(const float *red, int qty, int c) {
    float v = red[qty * kStrip + c];
    for (int w = 1; w < kWarps; ++w) {
        const float x = red[(w * kQ + qty) * kStrip + c];
        v = qty == 2 ? fmaxf(v, x) : qty == 3 ? fminf(v, x) : v + x;
    }
    return v;
}

// ---------------------------------------------------------------------------
// dense: pass over A, grid = (column strips, row splits)
// ---------------------------------------------------------------------------
template <bool VEC>
__global__ void __launch_bounds__(kThreads) feat_pass_kernel(const float *__restrict__ A, int64_t m, int64_t n,
                                                             int64_t lda, int raw, const float *__restrict__ G,
                                                             int64_t rows_per_split, float *__restrict__ part) {
    extern __shared__ float red[];               // kWarps x kQ x kStrip
    const int64_t cb = (int64_t)blockIdx.x * kStrip;
    const int64_t r0 = (int64_t)blockIdx.y * rows_per_split;
    strip_pass<VEC>(A, n, lda, raw, G, cb, r0, min(m, r0 + rows_per_split), red);
    __syncthreads();
    for (int e = threadIdx.x; e < kQ * kStrip; e += kThreads) {
        const int qty = e / kStrip, c = e % kStrip;
        const int64_t col = cb + c;
        if (col < n) part[((int64_t)blockIdx.y * n + col) * kQ + qty] = strip_combine(red, qty, c);
    }
}

// sum_i G[i, r] over all rows, in row-chunk order
__global__ void feat_gsum_kernel(const float *__restrict__ G, int64_t m, float *__restrict__ gsum) {
    __shared__ float red[kThreads / kSk][kSk];
    const int r = threadIdx.x % kSk, lane_row = threadIdx.x / kSk;
    float a = 0.f;
    for (int64_t i = lane_row; i < m; i += kThreads / kSk) a += G[i * kSk + r];
    red[lane_row][r] = a;
    __syncthreads();
    if (threadIdx.x < kSk) {
        float v = 0.f;
        for (int w = 0; w < kThreads / kSk; ++w) v += red[w][threadIdx.x];
        gsum[threadIdx.x] = v;
    }
}

// per column: combine the splits, finish the column; keep (c, q, x, S) in F's row and
// per-block sums of q and S[r]^2 in cpart
__global__ void feat_finish_kernel(const float *__restrict__ A, int64_t m, int64_t n, int raw,
                                   const float *__restrict__ part, int splits, const float *__restrict__ gsum,
                                   float *__restrict__ F, float *__restrict__ cpart) {
    __shared__ float red[kWarps][1 + kSk];
    const int64_t j = blockIdx.x * (int64_t)kThreads + threadIdx.x;
    float sums[1 + kSk];
#pragma unroll
    for (int e = 0; e <= kSk; ++e) sums[e] = 0.f;
    if (j < n) {
        float s1 = 0.f, s2 = 0.f, mx = -INFINITY, mn = INFINITY, Sd[kSk];
#pragma unroll
        for (int r = 0; r < kSk; ++r) Sd[r] = 0.f;
        for (int sp = 0; sp < splits; ++sp) {
            const float *p = part + ((int64_t)sp * n + j) * kQ;
            s1 += p[0];
            s2 += p[1];
            mx = fmaxf(mx, p[2]);
            mn = fminf(mn, p[3]);
#pragma unroll
            for (int r = 0; r < kSk; ++r) Sd[r] += p[4 + r];
        }
        float g[kSk];
#pragma unroll
        for (int r = 0; r < kSk; ++r) g[r] = gsum[r];
        const ColStats cs = finish_column(raw ? 0.f : A[j], s1, s2, mx, mn, Sd, g, m, raw);
        float *Fj = F + j * RPCA_MLP_FEATURES;
        Fj[0] = cs.q;
        Fj[1] = cs.c;
        Fj[2] = cs.x;
#pragma unroll
        for (int r = 0; r < kSk; ++r) Fj[3 + r] = cs.S[r];
        sums[0] = cs.q;
#pragma unroll
        for (int r = 0; r < kSk; ++r) sums[1 + r] = cs.S[r] * cs.S[r];
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int e = 0; e <= kSk; ++e) {
        float v = sums[e];
#pragma unroll
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][e] = v;
    }
    __syncthreads();
    if (threadIdx.x <= kSk) {
        float v = 0.f;
        for (int w = 0; w < kWarps; ++w) v += red[w][threadIdx.x];
        cpart[(int64_t)blockIdx.x * (1 + kSk) + threadIdx.x] = v;
    }
}

// stats[0] = qbar, stats[1 + r] = rho_r
__global__ void feat_stats_kernel(const float *__restrict__ cpart, int nblocks, int64_t n, float *__restrict__ stats) {
    if (threadIdx.x > kSk) return;
    float v = 0.f;
    for (int b = 0; b < nblocks; ++b) v += cpart[(int64_t)b * (1 + kSk) + threadIdx.x];
    v /= (float)n;
    stats[threadIdx.x] = threadIdx.x == 0 ? v : sqrtf(v);
}

__global__ void feat_write_kernel(int64_t m, int64_t n, const float *__restrict__ stats, float *__restrict__ F) {
    const int64_t j = blockIdx.x * (int64_t)kThreads + threadIdx.x;
    if (j >= n) return;
    float *Fj = F + j * RPCA_MLP_FEATURES;
    ColStats cs;
    cs.q = Fj[0];
    cs.c = Fj[1];
    cs.x = Fj[2];
#pragma unroll
    for (int r = 0; r < kSk; ++r) cs.S[r] = Fj[3 + r];
    float rho[kSk];
#pragma unroll
    for (int r = 0; r < kSk; ++r) rho[r] = stats[1 + r];
    write_features(Fj, cs, stats[0], rho, m, n);
}

struct FeatPlan {
    int splits = 1, strips = 1, fblocks = 1;
    int64_t rows_per_split = 1;
    size_t status = 0, G = 0, part = 0, gsum = 0, cpart = 0, stats = 0, total = 0;
};

FeatPlan feat_plan(int64_t m, int64_t n) {
    FeatPlan P;
    P.strips = (int)cdiv(n, (int64_t)kStrip);
    const int64_t want = cdiv(4LL * num_sms(), (int64_t)P.strips);
    P.splits = (int)std::max<int64_t>(1, std::min<int64_t>(want, cdiv(m, (int64_t)256)));
    P.rows_per_split = cdiv(m, (int64_t)P.splits);
    P.splits = (int)cdiv(m, P.rows_per_split);
    P.fblocks = (int)cdiv(n, (int64_t)kThreads);
    auto a256 = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t off = 0;
    P.status = off; off = a256(off + sizeof(DevStatus));
    P.G = off; off = a256(off + (size_t)m * kSk * 4);
    P.part = off; off = a256(off + (size_t)P.splits * n * kQ * 4);
    P.gsum = off; off = a256(off + kSk * 4);
    P.cpart = off; off = a256(off + (size_t)P.fblocks * (1 + kSk) * 4);
    P.stats = off; off = a256(off + (1 + kSk) * 4);
    P.total = off;
    return P;
}

// ---------------------------------------------------------------------------
// batched: one CTA per matrix; G (max_m x 8) precomputed, shared by all items
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads, 2) feat_batched_kernel(int count, const rpca_mat_desc *__restrict__ descs,
                                                                int raw, const float *__restrict__ G,
                                                                int64_t max_m,
                                                                const int64_t *__restrict__ col_offsets,
                                                                float *__restrict__ F) {
    extern __shared__ float red[];               // kWarps x kQ x kStrip
    __shared__ float gpart[kThreads / kSk][kSk];
    __shared__ float wred[kWarps][1 + kSk];
    __shared__ float tot[1 + kSk];
    __shared__ float gsum_s[kSk];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int item = blockIdx.x; item < count; item += gridDim.x) {
        const rpca_mat_desc dsc = descs[item];
        const int64_t m = dsc.m, n = dsc.n, lda = dsc.lda;
        if (!dsc.A || m < 1 || n < 1 || lda < n || m > max_m) continue;     // uniform across the CTA
        const float *A = dsc.A;
        float *Fi = F + col_offsets[item] * RPCA_MLP_FEATURES;
        // sum_i G[i, r] over this item's rows
        {
            const int r = tid % kSk, rr = tid / kSk;
            float a = 0.f;
            for (int64_t i = rr; i < m; i += kThreads / kSk) a += G[i * kSk + r];
            gpart[rr][r] = a;
            __syncthreads();
            if (tid < kSk) {
                float v = 0.f;
                for (int w = 0; w < kThreads / kSk; ++w) v += gpart[w][tid];
                gsum_s[tid] = v;
            }
            __syncthreads();
        }
        float g[kSk];
#pragma unroll
        for (int r = 0; r < kSk; ++r) g[r] = gsum_s[r];
        const bool vec = (reinterpret_cast<uintptr_t>(A) & 15u) == 0 && lda % 4 == 0;
        float qsum = 0.f, ssq[kSk];
#pragma unroll
        for (int r = 0; r < kSk; ++r) ssq[r] = 0.f;
        for (int64_t cb = 0; cb < n; cb += kStrip) {
            if (vec) strip_pass<true>(A, n, lda, raw, G, cb, 0, m, red);
            else strip_pass<false>(A, n, lda, raw, G, cb, 0, m, red);
            __syncthreads();
            const int64_t col = cb + tid;
            if (tid < kStrip && col < n) {
                float Sd[kSk];
#pragma unroll
                for (int r = 0; r < kSk; ++r) Sd[r] = strip_combine(red, 4 + r, tid);
                const ColStats cs = finish_column(raw ? 0.f : A[col], strip_combine(red, 0, tid),
                                                  strip_combine(red, 1, tid), strip_combine(red, 2, tid),
                                                  strip_combine(red, 3, tid), Sd, g, m, raw);
                float *Fj = Fi + col * RPCA_MLP_FEATURES;
                Fj[0] = cs.q;
                Fj[1] = cs.c;
                Fj[2] = cs.x;
#pragma unroll
                for (int r = 0; r < kSk; ++r) Fj[3 + r] = cs.S[r];
                qsum += cs.q;
#pragma unroll
                for (int r = 0; r < kSk; ++r) ssq[r] = fmaf(cs.S[r], cs.S[r], ssq[r]);
            }
            __syncthreads();
        }
        // CTA totals: qbar and rho
        {
            float v[1 + kSk];
            v[0] = qsum;
#pragma unroll
            for (int r = 0; r < kSk; ++r) v[1 + r] = ssq[r];
#pragma unroll
            for (int e = 0; e <= kSk; ++e) {
#pragma unroll
                for (int o = 16; o; o >>= 1) v[e] += __shfl_xor_sync(0xffffffffu, v[e], o);
                if (lane == 0) wred[warp][e] = v[e];
            }
        }
        __syncthreads();
        if (tid <= kSk) {
            float v = 0.f;
            for (int w = 0; w < kWarps; ++w) v += wred[w][tid];
            v /= (float)n;
            tot[tid] = tid == 0 ? v : sqrtf(v);
        }
        __syncthreads();
        float rho[kSk];
#pragma unroll
        for (int r = 0; r < kSk; ++r) rho[r] = tot[1 + r];
        const float qbar = tot[0];
        for (int64_t col = tid; col < n; col += kThreads) {
            float *Fj = Fi + col * RPCA_MLP_FEATURES;
            ColStats cs;
            cs.q = Fj[0];
            cs.c = Fj[1];
            cs.x = Fj[2];
#pragma unroll
            for (int r = 0; r < kSk; ++r) cs.S[r] = Fj[3 + r];
            write_features(Fj, cs, qbar, rho, m, n);
        }
        __syncthreads();
    }
}

}  // namespace

size_t features_workspace_size(int64_t m, int64_t n) { return feat_plan(m, n).total; }

int launch_features(const float *A, int64_t m, int64_t n, int64_t lda, int raw, uint64_t seed, float *F, void *ws,
                    cudaStream_t s) {
    const FeatPlan P = feat_plan(m, n);
    char *base = static_cast<char *>(ws);
    float *G = reinterpret_cast<float *>(base + P.G);
    float *part = reinterpret_cast<float *>(base + P.part);
    float *gsum = reinterpret_cast<float *>(base + P.gsum);
    float *cpart = reinterpret_cast<float *>(base + P.cpart);
    float *stats = reinterpret_cast<float *>(base + P.stats);
    RPCA_TRY(launch_omega(m, kSk, seed, 2, nullptr, G, kSk, s));
    const dim3 grid(P.strips, P.splits);
    const size_t smem = (size_t)kWarps * kQ * kStrip * sizeof(float);
    const bool vec = (reinterpret_cast<uintptr_t>(A) & 15u) == 0 && lda % 4 == 0;
    for (auto k : {feat_pass_kernel<true>, feat_pass_kernel<false>})
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return RPCA_ERR_CUDA;
    if (vec) feat_pass_kernel<true><<<grid, kThreads, smem, s>>>(A, m, n, lda, raw, G, P.rows_per_split, part);
    else feat_pass_kernel<false><<<grid, kThreads, smem, s>>>(A, m, n, lda, raw, G, P.rows_per_split, part);
    RPCA_CHECK_LAUNCH();
    feat_gsum_kernel<<<1, kThreads, 0, s>>>(G, m, gsum);
    RPCA_CHECK_LAUNCH();
    feat_finish_kernel<<<P.fblocks, kThreads, 0, s>>>(A, m, n, raw, part, P.splits, gsum, F, cpart);
    RPCA_CHECK_LAUNCH();
    feat_stats_kernel<<<1, 32, 0, s>>>(cpart, P.fblocks, n, stats);
    RPCA_CHECK_LAUNCH();
    feat_write_kernel<<<P.fblocks, kThreads, 0, s>>>(m, n, stats, F);
    RPCA_CHECK_LAUNCH();
    return RPCA_OK;
}

}  // namespace rpca

using namespace rpca;

extern "C" size_t rpca_features_workspace_size(int64_t m, int64_t n) {
    if (m < 1 || n < 1) return 0;
    return features_workspace_size(m, n);
}

extern "C" int rpca_sketch_features(const float *A, int64_t m, int64_t n, int64_t lda, int32_t raw, uint64_t seed,
                                    float *F, void *ws, size_t ws_bytes, rpca_stream_t stream) {
    if (!A || !F || m < 1 || n < 1 || lda < n) return RPCA_ERR_INVALID_ARG;
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0 || ws_bytes < features_workspace_size(m, n))
        return RPCA_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(ws, 0, sizeof(DevStatus), s) != cudaSuccess) return RPCA_ERR_CUDA;
    return launch_features(A, m, n, lda, raw ? 1 : 0, seed, F, ws, s);
}

extern "C" size_t rpca_batched_features_workspace_size(int64_t max_m) {
    if (max_m < 1) return 0;
    return ((size_t)max_m * kSk * sizeof(float) + 255) & ~(size_t)255;
}

extern "C" int rpca_batched_features(int32_t count, const rpca_mat_desc *descs, int64_t max_m, int32_t raw,
                                     uint64_t seed, const int64_t *col_offsets, float *F, void *ws, size_t ws_bytes,
                                     rpca_stream_t stream) {
    if (count < 0 || max_m < 1 || (count > 0 && (!descs || !col_offsets || !F))) return RPCA_ERR_INVALID_ARG;
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0 || ws_bytes < rpca_batched_features_workspace_size(max_m))
        return RPCA_ERR_WORKSPACE;
    if (count == 0) return RPCA_OK;
    cudaStream_t s = (cudaStream_t)stream;
    float *G = static_cast<float *>(ws);
    RPCA_TRY(launch_omega(max_m, kSk, seed, 2, nullptr, G, kSk, s));
    const size_t smem = (size_t)kWarps * kQ * kStrip * sizeof(float);
    if (cudaFuncSetAttribute(feat_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return RPCA_ERR_CUDA;
    const int grid = std::min<int>(count, 2 * num_sms());
    feat_batched_kernel<<<grid, kThreads, smem, s>>>(count, descs, raw ? 1 : 0, G, max_m, col_offsets, F);
    RPCA_CHECK_LAUNCH();
    return RPCA_OK;
}

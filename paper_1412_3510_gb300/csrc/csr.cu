// Sparse A in CSR form.  Section 5 notes that the same code serves dense and
// sparse A: only the two products change.  A X is a gather SpMM over the rows
// of A; A^T Q is the same SpMM over the rows of A^T, which is built once per
// call by a stable radix sort of the nonzeros by column (no atomics anywhere,
// so every result is deterministic).
//
// SpMM: a group of 8, 16 or 32 lanes per row (by the block width), lanes across
// the l-wide block in float4 (the block operand is read from L2 row by row), four
// nonzeros per step, several rows per warp so that many gathers are in flight.  Rows with more than kHeavy nonzeros (power-law degree
// distributions have rows with ~1e5 of them) are cut into chunks of kHeavy
// nonzeros, one warp per chunk writing a partial row, and a third kernel adds
// each heavy row's partials in chunk order.
#include "pipeline.cuh"
#include "resid.cuh"
#include "timing.cuh"

namespace rpca {

namespace {

constexpr int kHeavy = 256;
constexpr int kTile = 4096;            // radix sort: nonzeros per block (8 warps x 512)
constexpr int kSortThreads = 256;

// row_of[p] = r for every nonzero p of row r: one warp per row, lanes across its range
// (coalesced stores).  Ranges are clamped to [0, nnz); positions that no row covers (a
// malformed row_ptr, reported by csr_check_kernel) keep the zero the caller wrote.
__global__ void __launch_bounds__(256) row_expand_kernel(const int32_t *__restrict__ ptr, int64_t rows, int64_t nnz,
                                                         int32_t *__restrict__ row_of) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = wid; r < rows; r += nw) {
        const int64_t p0 = max((int64_t)ptr[r], (int64_t)0), p1 = min((int64_t)ptr[r + 1], nnz);
        for (int64_t p = p0 + lane; p < p1; p += 32) row_of[p] = (int32_t)r;
    }
}

__global__ void copy_i32_kernel(const int32_t *__restrict__ a, int32_t *__restrict__ b, int64_t n) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) b[p] = a[p];
}
__global__ void copy_f32_kernel(const float *__restrict__ a, float *__restrict__ b, int64_t n) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) b[p] = a[p];
}

// hist[bin * nblocks + block] = number of keys of the block whose digit is bin
__global__ void __launch_bounds__(kSortThreads)
radix_hist_kernel(const int32_t *__restrict__ keys, int64_t count, int shift, int32_t *__restrict__ hist, int nblocks) {
    __shared__ int h[256];
    for (int b = threadIdx.x; b < 256; b += blockDim.x) h[b] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTile;
    for (int e = threadIdx.x; e < kTile; e += blockDim.x) {
        const int64_t i = base + e;
        if (i < count) atomicAdd(&h[((uint32_t)keys[i] >> shift) & 255u], 1);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[(int64_t)b * nblocks + blockIdx.x] = h[b];
}

// In-place exclusive scan of `total` counts in three launches: per-tile sums, a
// scan of the tile sums (one CTA), and per-tile scans with the tile offsets.
constexpr int kScanThreads = 256, kScanPer = 16, kScanTile = kScanThreads * kScanPer;

__global__ void __launch_bounds__(kScanThreads) scan_sums_kernel(const int32_t *__restrict__ data, int64_t total,
                                                                 int64_t *__restrict__ sums) {
    __shared__ int64_t red[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t s = 0;
    for (int e = threadIdx.x; e < kScanTile; e += kScanThreads) {
        const int64_t i = base + e;
        if (i < total) s += data[i];
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t t = 0;
        for (int w = 0; w < kScanThreads / 32; ++w) t += red[w];
        sums[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(1024) scan_top_kernel(int64_t *__restrict__ sums, int64_t n) {
    __shared__ int64_t part[1024];
    const int64_t per = (n + blockDim.x - 1) / blockDim.x;
    const int64_t b = threadIdx.x * per, e = min(n, b + per);
    int64_t s = 0;
    for (int64_t i = b; i < e; ++i) s += sums[i];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t run = 0;
        for (int t = 0; t < (int)blockDim.x; ++t) { const int64_t v = part[t]; part[t] = run; run += v; }
    }
    __syncthreads();
    int64_t run = part[threadIdx.x];
    for (int64_t i = b; i < e; ++i) { const int64_t v = sums[i]; sums[i] = run; run += v; }
}

// thread t scans kScanPer consecutive entries of the tile
__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(int32_t *__restrict__ data, int64_t total,
                                                                  const int64_t *__restrict__ sums) {
    __shared__ int64_t wsum[kScanThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
    int32_t v[kScanPer];
    int64_t own = 0;
#pragma unroll
    for (int u = 0; u < kScanPer; ++u) {
        v[u] = base + u < total ? data[base + u] : 0;
        own += v[u];
    }
    int64_t incl = own;                               // inclusive scan over the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    int64_t before = sums[blockIdx.x] + incl - own;
    for (int w = 0; w < warp; ++w) before += wsum[w];
#pragma unroll
    for (int u = 0; u < kScanPer; ++u) {
        if (base + u < total) data[base + u] = (int32_t)before;
        before += v[u];
    }
}

int64_t scan_tiles(int64_t total) { return std::max<int64_t>(1, cdiv(total, (int64_t)kScanTile)); }

int launch_scan(int32_t *data, int64_t total, int64_t *sums, cudaStream_t s) {
    if (total <= 0) return RPCA_OK;
    const int64_t tiles = scan_tiles(total);
    scan_sums_kernel<<<(unsigned)tiles, kScanThreads, 0, s>>>(data, total, sums);
    RPCA_CHECK_LAUNCH();
    scan_top_kernel<<<1, 1024, 0, s>>>(sums, tiles);
    RPCA_CHECK_LAUNCH();
    scan_apply_kernel<<<(unsigned)tiles, kScanThreads, 0, s>>>(data, total, sums);
    RPCA_CHECK_LAUNCH();
    return RPCA_OK;
}

// stable scatter by digit: warp w of a block handles nonzeros [block*kTile + 512 w, +512) in order
__global__ void __launch_bounds__(kSortThreads)
radix_scatter_kernel(const int32_t *__restrict__ kin, const int32_t *__restrict__ rin, const float *__restrict__ vin,
                     int64_t count, int shift, const int32_t *__restrict__ offs, int nblocks,
                     int32_t *__restrict__ kout, int32_t *__restrict__ rout, float *__restrict__ vout) {
    __shared__ int wc[8][256];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int b = lane; b < 256; b += 32) wc[warp][b] = 0;
    __syncwarp();
    const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)warp * (kTile / 8);
    for (int step = 0; step < kTile / 8 / 32; ++step) {
        const int64_t i = base + step * 32 + lane;
        const int bin = i < count ? (int)(((uint32_t)kin[i] >> shift) & 255u) : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, bin);
        if (bin >= 0 && lane == __ffs(peers) - 1) wc[warp][bin] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    for (int b = threadIdx.x; b < 256; b += blockDim.x) {
        int run = offs[(int64_t)b * nblocks + blockIdx.x];
        for (int w = 0; w < 8; ++w) { const int t = wc[w][b]; wc[w][b] = run; run += t; }
    }
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    for (int step = 0; step < kTile / 8 / 32; ++step) {
        const int64_t i = base + step * 32 + lane;
        const int bin = i < count ? (int)(((uint32_t)kin[i] >> shift) & 255u) : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, bin);
        if (bin >= 0) {
            const int dest = wc[warp][bin] + __popc(peers & lt);
            kout[dest] = kin[i];
            rout[dest] = rin[i];
            vout[dest] = vin[i];
        }
        __syncwarp();
        if (bin >= 0 && lane == __ffs(peers) - 1) wc[warp][bin] += __popc(peers);
        __syncwarp();
    }
}

// colptr[c] = first position whose key >= c (c = 0..n)
__global__ void colptr_kernel(const int32_t *__restrict__ keys, int64_t nnz, int64_t n, int32_t *__restrict__ colptr) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c <= n; c += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = nnz;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if ((int64_t)keys[mid] < c) lo = mid + 1; else hi = mid;
        }
        colptr[c] = (int32_t)lo;
    }
}

// heavy-row chunk counts: cnt[r] = deg(r) > kHeavy ? ceil(deg / kHeavy) : 0, cnt[rows] = 0
__global__ void chunk_count_kernel(const int32_t *__restrict__ ptr, int64_t rows, int32_t *__restrict__ cnt) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r <= rows; r += (int64_t)gridDim.x * blockDim.x) {
        int32_t c = 0;
        if (r < rows) {
            const int32_t d = max(ptr[r + 1] - ptr[r], 0);
            c = d > kHeavy ? (d + kHeavy - 1) / kHeavy : 0;
        }
        cnt[r] = c;
    }
}

// after the exclusive scan, cnt[r] = first chunk of row r; table[chunk] = (row, q)
__global__ void chunk_table_kernel(const int32_t *__restrict__ ptr, const int32_t *__restrict__ first, int64_t rows,
                                   int2 *__restrict__ table, int64_t max_chunks) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = first[r + 1] - first[r];
        for (int q = 0; q < c; ++q)
            if ((int64_t)first[r] + q < max_chunks) table[first[r] + q] = make_int2((int)r, q);
    }
}

// Input check: row_ptr[0] = 0, nondecreasing, row_ptr[m] = nnz; 0 <= col_idx < n.
// A violation is recorded as RPCA_ERR_INVALID_ARG; the SpMM kernels clamp and
// skip out-of-range entries, so nothing is read out of bounds either way.
__global__ void csr_check_kernel(const int32_t *__restrict__ ptr, const int32_t *__restrict__ idx, int64_t m,
                                 int64_t n, int64_t nnz, DevStatus *__restrict__ st) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x)
        if (ptr[r + 1] < ptr[r] || (r == 0 && ptr[0] != 0) || (r == m - 1 && (int64_t)ptr[m] != nnz))
            dev_fail(st, RPCA_ERR_INVALID_ARG);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x)
        if (idx[p] < 0 || (int64_t)idx[p] >= n) dev_fail(st, RPCA_ERR_INVALID_ARG);
}

// acc[q] += sum_{p0 <= p < p1} val[p] X[idx[p]][c0 + lane + 32 q], eight nonzeros per step;
// entries with a column outside [0, cols) contribute nothing.
__device__ __forceinline__ void row_dot(const int32_t *__restrict__ idx, const float *__restrict__ val, int32_t p0,
                                        int32_t p1, int64_t cols, const float *__restrict__ X, int lp, int c0,
                                        int lane, float (&acc)[4]) {
    int32_t p = p0;
    for (; p + 8 <= p1; p += 8) {
        int32_t j[8];
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            j[u] = __ldg(idx + p + u);
            v[u] = __ldg(val + p + u);
            if ((uint32_t)j[u] >= (uint32_t)cols) { j[u] = 0; v[u] = 0.f; }
        }
        float x[8][4];
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int c = c0 + lane + 32 * q;
                x[u][q] = c < lp ? __ldg(X + (int64_t)j[u] * lp + c) : 0.f;
            }
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = fmaf(v[u], x[u][q], acc[q]);
    }
    for (; p < p1; ++p) {
        const int32_t jj = __ldg(idx + p);
        if ((uint32_t)jj >= (uint32_t)cols) continue;
        const float vv = __ldg(val + p);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int c = c0 + lane + 32 * q;
            if (c < lp) acc[q] = fmaf(vv, __ldg(X + (int64_t)jj * lp + c), acc[q]);
        }
    }
}

// light rows: Y[r] = sum_p val[p] X[idx[p]] (heavy rows are skipped)
__global__ void __launch_bounds__(256)
spmm_light_kernel(const int32_t *__restrict__ ptr, const int32_t *__restrict__ idx, const float *__restrict__ val,
                  int64_t rows, int64_t cols, int64_t nnz, const float *__restrict__ X, int lp, float *__restrict__ Y) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = wid; r < rows; r += nw) {
        const int32_t p0 = max(ptr[r], 0), p1 = min((int64_t)ptr[r + 1], nnz);
        if (p1 - p0 > kHeavy) continue;
        for (int c0 = 0; c0 < lp; c0 += 128) {
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
            row_dot(idx, val, p0, p1, cols, X, lp, c0, lane, acc);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int c = lane + 32 * q;
                if (c0 + c < lp) Y[r * lp + c0 + c] = acc[q];
            }
        }
    }
}

// a0, a1 (two float4 of a G-lane group's share of the l-wide row: columns 4 sub and
// 4 (sub + G)) += sum_{p0 <= p < p1} val[p] X[idx[p]], four nonzeros per step;
// entries with a column outside [0, cols) contribute nothing.
template <int G>
__device__ __forceinline__ void group_dot(const int32_t *__restrict__ idx, const float *__restrict__ val, int32_t p0,
                                          int32_t p1, int64_t cols, const float4 *__restrict__ X4, int nv, int sub,
                                          bool c0ok, bool c1ok, float4 &a0, float4 &a1) {
    // Software-pipelined: the next step's indices and values load while this step's
    // block rows are gathered, so a step waits for one memory round trip, not two.
    // Nonzeros are accumulated in order p0, p0 + 1, ... (as a plain loop would).
    int32_t jn[4];
    float vn[4];
    auto fetch = [&](int32_t p) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const bool in = p + u < p1;
            jn[u] = in ? __ldg(idx + p + u) : 0;
            vn[u] = in ? __ldg(val + p + u) : 0.f;
        }
    };
    if (p0 < p1) fetch(p0);
    for (int32_t p = p0; p < p1; p += 4) {
        const int cnt = min(4, p1 - p);
        int32_t j[4];
        float v[4];
        bool ok[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            j[u] = jn[u];
            v[u] = vn[u];
            ok[u] = u < cnt && (uint32_t)j[u] < (uint32_t)cols;
        }
        float4 x0[4], x1[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float4 *xr = X4 + (int64_t)(ok[u] ? j[u] : 0) * nv;
            x0[u] = (ok[u] && c0ok) ? __ldg(xr + sub) : make_float4(0.f, 0.f, 0.f, 0.f);
            x1[u] = (ok[u] && c1ok) ? __ldg(xr + sub + G) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        if (p + 4 < p1) fetch(p + 4);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (!ok[u]) continue;
            a0.x = fmaf(v[u], x0[u].x, a0.x); a0.y = fmaf(v[u], x0[u].y, a0.y);
            a0.z = fmaf(v[u], x0[u].z, a0.z); a0.w = fmaf(v[u], x0[u].w, a0.w);
            a1.x = fmaf(v[u], x1[u].x, a1.x); a1.y = fmaf(v[u], x1[u].y, a1.y);
            a1.z = fmaf(v[u], x1[u].z, a1.z); a1.w = fmaf(v[u], x1[u].w, a1.w);
        }
    }
}

// Light rows in order of degree bucket (0, 1, 2-3, 4-7, ..., 129-256 nonzeros), so that
// the rows sharing a warp have lengths within a factor of two: with power-law degrees a
// warp would otherwise run as long as the longest of its rows.  The order within a
// bucket comes from atomics and varies, which changes nothing: every row's sum is its
// own.  Heavy rows are left out (their chunks have their own kernels).
constexpr int kBuckets = 10;
constexpr int kBucketRows = 1024;             // rows per CTA of the bucket kernels

__device__ __forceinline__ int light_bucket(const int32_t *__restrict__ ptr, int64_t r, int64_t nnz) {
    const int32_t p0 = max(ptr[r], 0), p1 = (int32_t)min((int64_t)ptr[r + 1], nnz);
    const int d = p1 - p0;
    if (d > kHeavy) return -1;
    return d <= 0 ? 0 : 32 - __clz(d);
}

// cnt[b] += number of light rows in bucket b (cnt zeroed by the caller)
__global__ void __launch_bounds__(256) bucket_count_kernel(const int32_t *__restrict__ ptr, int64_t rows, int64_t nnz,
                                                           int32_t *__restrict__ cnt) {
    __shared__ int h[kBuckets];
    if (threadIdx.x < kBuckets) h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t r0 = (int64_t)blockIdx.x * kBucketRows;
    for (int e = threadIdx.x; e < kBucketRows; e += blockDim.x) {
        const int64_t r = r0 + e;
        if (r < rows) {
            const int b = light_bucket(ptr, r, nnz);
            if (b >= 0) atomicAdd(&h[b], 1);
        }
    }
    __syncthreads();
    if (threadIdx.x < kBuckets && h[threadIdx.x]) atomicAdd(&cnt[threadIdx.x], h[threadIdx.x]);
}

// cnt -> exclusive offsets in cur[0..kBuckets-1], the number of light rows in cur[kBuckets]
__global__ void bucket_scan_kernel(const int32_t *__restrict__ cnt, int32_t *__restrict__ cur) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int32_t run = 0;
        for (int b = 0; b < kBuckets; ++b) { cur[b] = run; run += cnt[b]; }
        cur[kBuckets] = run;
    }
}

// perm[cur[b]++ ...] = the light rows of bucket b (one global atomic per CTA and bucket)
__global__ void __launch_bounds__(256) bucket_scatter_kernel(const int32_t *__restrict__ ptr, int64_t rows, int64_t nnz,
                                                             int32_t *__restrict__ cur, int32_t *__restrict__ perm) {
    __shared__ int h[kBuckets], base[kBuckets];
    if (threadIdx.x < kBuckets) h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t r0 = (int64_t)blockIdx.x * kBucketRows;
    int bk[kBucketRows / 256], rk[kBucketRows / 256];
#pragma unroll
    for (int u = 0; u < kBucketRows / 256; ++u) {
        const int64_t r = r0 + threadIdx.x + 256 * u;
        bk[u] = r < rows ? light_bucket(ptr, r, nnz) : -1;
        rk[u] = bk[u] >= 0 ? atomicAdd(&h[bk[u]], 1) : 0;
    }
    __syncthreads();
    if (threadIdx.x < kBuckets) base[threadIdx.x] = h[threadIdx.x] ? atomicAdd(&cur[threadIdx.x], h[threadIdx.x]) : 0;
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kBucketRows / 256; ++u)
        if (bk[u] >= 0) perm[base[bk[u]] + rk[u]] = (int32_t)(r0 + threadIdx.x + 256 * u);
}

// light rows with several rows per warp: a group of G lanes per row, every warp keeping
// (32 / G) x 4 x 2 float4 gathers in flight.  Needs lp % 4 == 0 and lp <= 8 G; heavy
// rows are skipped.
template <int G>
__global__ void __launch_bounds__(256, 4)
spmm_light_group_kernel(const int32_t *__restrict__ ptr, const int32_t *__restrict__ idx,
                        const float *__restrict__ val, int64_t rows, int64_t cols, int64_t nnz,
                        const float *__restrict__ X, int lp, float *__restrict__ Y, const int32_t *__restrict__ perm,
                        const int32_t *__restrict__ nlight) {
    constexpr int R = 32 / G;                  // rows per warp
    const int lane = threadIdx.x & 31, sub = lane % G, grp = lane / G;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int nv = lp >> 2;
    const bool c0ok = sub < nv, c1ok = sub + G < nv;
    const float4 *X4 = reinterpret_cast<const float4 *>(X);
    const int64_t nl = min((int64_t)*nlight, rows);
    for (int64_t rb = wid * R; rb < nl; rb += nw * R) {
        const int64_t q = rb + grp;
        const int64_t r = q < nl ? (int64_t)perm[q] : rows;
        int32_t p0 = 0, p1 = 0;
        bool write = false;
        if (r >= 0 && r < rows) {
            p0 = max(ptr[r], 0);
            p1 = (int32_t)min((int64_t)ptr[r + 1], nnz);
            write = p1 - p0 <= kHeavy;
            if (!write) p1 = p0;
        }
        float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0;
        group_dot<G>(idx, val, p0, p1, cols, X4, nv, sub, c0ok, c1ok, a0, a1);
        if (write) {
            float4 *yr = reinterpret_cast<float4 *>(Y) + r * nv;
            if (c0ok) yr[sub] = a0;
            if (c1ok) yr[sub + G] = a1;
        }
    }
}

// heavy chunks, a G-lane group per chunk: part[chunk] = sum over the chunk's nonzeros
template <int G>
__global__ void __launch_bounds__(256, 4)
spmm_heavy_group_kernel(const int32_t *__restrict__ ptr, const int32_t *__restrict__ idx,
                        const float *__restrict__ val, const int32_t *__restrict__ first, int64_t rows,
                        int64_t cols, int64_t nnz, const int2 *__restrict__ table, int64_t max_chunks,
                        const float *__restrict__ X, int lp, float *__restrict__ part) {
    constexpr int R = 32 / G;
    const int lane = threadIdx.x & 31, sub = lane % G, grp = lane / G;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int nv = lp >> 2;
    const bool c0ok = sub < nv, c1ok = sub + G < nv;
    const float4 *X4 = reinterpret_cast<const float4 *>(X);
    const int64_t nchunks = min((int64_t)first[rows], max_chunks);
    for (int64_t cb = wid * R; cb < nchunks; cb += nw * R) {
        const int64_t ch = cb + grp;
        int32_t p0 = 0, p1 = 0;
        if (ch < nchunks) {
            const int2 rq = table[ch];
            p0 = max(ptr[rq.x] + rq.y * kHeavy, 0);
            p1 = (int32_t)min(min((int64_t)ptr[rq.x + 1], (int64_t)p0 + kHeavy), nnz);
        }
        float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0;
        group_dot<G>(idx, val, p0, p1, cols, X4, nv, sub, c0ok, c1ok, a0, a1);
        if (ch < nchunks) {
            float4 *pr = reinterpret_cast<float4 *>(part) + ch * nv;
            if (c0ok) pr[sub] = a0;
            if (c1ok) pr[sub + G] = a1;
        }
    }
}

// heavy chunks: part[chunk] = sum over the chunk's nonzeros
__global__ void __launch_bounds__(256)
spmm_heavy_kernel(const int32_t *__restrict__ ptr, const int32_t *__restrict__ idx, const float *__restrict__ val,
                  const int32_t *__restrict__ first, int64_t rows, int64_t cols, int64_t nnz,
                  const int2 *__restrict__ table, int64_t max_chunks,
                  const float *__restrict__ X, int lp, float *__restrict__ part) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nchunks = min((int64_t)first[rows], max_chunks);
    for (int64_t ch = wid; ch < nchunks; ch += nw) {
        const int2 rq = table[ch];
        const int32_t p0 = max(ptr[rq.x] + rq.y * kHeavy, 0);
        const int32_t p1 = (int32_t)min(min((int64_t)ptr[rq.x + 1], (int64_t)p0 + kHeavy), nnz);
        for (int c0 = 0; c0 < lp; c0 += 128) {
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
            row_dot(idx, val, p0, p1, cols, X, lp, c0, lane, acc);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int c = lane + 32 * q;
                if (c0 + c < lp) part[ch * lp + c0 + c] = acc[q];
            }
        }
    }
}

// heavy rows: Y[r] = sum of its chunk partials, one CTA per row (found through the chunk
// table: the row's first chunk, q = 0).  Warp w sums chunks w, w + 8, ... with four
// interleaved partial sums; the eight warp sums are added in warp order (a fixed tree,
// so the result is deterministic).  A row of hundreds of chunks then has 32 loads in
// flight per column instead of one warp walking them.
constexpr int kReduceWarps = 8;

__global__ void __launch_bounds__(kReduceWarps * 32)
spmm_heavy_reduce_kernel(const int32_t *__restrict__ first, const int2 *__restrict__ table, int64_t rows,
                         int64_t max_chunks, const float *__restrict__ part, int lp, float *__restrict__ Y) {
    __shared__ float ws[kReduceWarps][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t nchunks = min((int64_t)first[rows], max_chunks);
    for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const int2 rq = table[ch];
        if (rq.y != 0) continue;                        // CTA-uniform
        const int64_t r = rq.x;
        const int64_t c0 = first[r], c1 = min((int64_t)first[r + 1], max_chunks);
        for (int cb = 0; cb < lp; cb += 32) {
            const int c = cb + lane;
            float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
            if (c < lp) {
                int64_t k = c0 + warp;
                for (; k + 3 * kReduceWarps < c1; k += 4 * kReduceWarps) {
                    s0 += part[k * lp + c];
                    s1 += part[(k + kReduceWarps) * lp + c];
                    s2 += part[(k + 2 * kReduceWarps) * lp + c];
                    s3 += part[(k + 3 * kReduceWarps) * lp + c];
                }
                if (k < c1) s0 += part[k * lp + c];
                if (k + kReduceWarps < c1) s1 += part[(k + kReduceWarps) * lp + c];
                if (k + 2 * kReduceWarps < c1) s2 += part[(k + 2 * kReduceWarps) * lp + c];
            }
            ws[warp][lane] = (s0 + s1) + (s2 + s3);
            __syncthreads();
            if (warp == 0 && c < lp) {
                float t = ws[0][lane];
#pragma unroll
                for (int w = 1; w < kReduceWarps; ++w) t += ws[w][lane];
                Y[r * lp + c] = t;
            }
            __syncthreads();
        }
    }
}

int grid_for(int64_t work, int per_block) {
    return (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(work, per_block), (int64_t)num_sms() * 16));
}

// Storage of one SpMM operand (a CSR matrix) and its heavy-row plan.
struct Spmm {
    const int32_t *ptr = nullptr, *idx = nullptr;
    const float *val = nullptr;
    int64_t rows = 0, cols = 0, nnz = 0, max_chunks = 0;
    int32_t *first = nullptr;      // rows + 1
    int32_t *perm = nullptr;       // rows: light rows by degree bucket
    int32_t *bk = nullptr;         // 2 kBuckets + 1: bucket counts, offsets / the number of light rows
    int2 *table = nullptr;         // max_chunks
    float *part = nullptr;         // max_chunks x max_lp
    int64_t *scan_tmp = nullptr;   // scan_tiles(rows + 1)

    int plan(cudaStream_t s) const {
        chunk_count_kernel<<<grid_for(rows + 1, 256), 256, 0, s>>>(ptr, rows, first);
        RPCA_CHECK_LAUNCH();
        const int64_t bblocks = std::max<int64_t>(1, cdiv(rows, kBucketRows));
        if (cudaMemsetAsync(bk, 0, (2 * kBuckets + 1) * sizeof(int32_t), s) != cudaSuccess) return RPCA_ERR_CUDA;
        bucket_count_kernel<<<(unsigned)bblocks, 256, 0, s>>>(ptr, rows, nnz, bk);
        RPCA_CHECK_LAUNCH();
        bucket_scan_kernel<<<1, 32, 0, s>>>(bk, bk + kBuckets);
        RPCA_CHECK_LAUNCH();
        bucket_scatter_kernel<<<(unsigned)bblocks, 256, 0, s>>>(ptr, rows, nnz, bk + kBuckets, perm);
        RPCA_CHECK_LAUNCH();
        // bucket_scatter advanced the offsets by the counts: bk[2 kBuckets] still holds the total
        RPCA_TRY(launch_scan(first, rows + 1, scan_tmp, s));
        if (max_chunks > 0) {
            chunk_table_kernel<<<grid_for(rows, 256), 256, 0, s>>>(ptr, first, rows, table, max_chunks);
            RPCA_CHECK_LAUNCH();
        }
        return RPCA_OK;
    }
    int run(const float *X, int lp, float *Y, cudaStream_t s) const {
        const bool vec = lp % 4 == 0 && (reinterpret_cast<uintptr_t>(X) & 15u) == 0 &&
                         (reinterpret_cast<uintptr_t>(Y) & 15u) == 0;
        if (vec && lp <= 64) {
            spmm_light_group_kernel<8><<<grid_for(rows * 8, 256), 256, 0, s>>>(ptr, idx, val, rows, cols, nnz, X, lp, Y, perm, bk + 2 * kBuckets);
        } else if (vec && lp <= 128) {
            spmm_light_group_kernel<16><<<grid_for(rows * 16, 256), 256, 0, s>>>(ptr, idx, val, rows, cols, nnz, X, lp, Y, perm, bk + 2 * kBuckets);
        } else if (vec && lp <= 256) {
            spmm_light_group_kernel<32><<<grid_for(rows * 32, 256), 256, 0, s>>>(ptr, idx, val, rows, cols, nnz, X, lp, Y, perm, bk + 2 * kBuckets);
        } else {
            spmm_light_kernel<<<grid_for(rows * 32, 256), 256, 0, s>>>(ptr, idx, val, rows, cols, nnz, X, lp, Y);
        }
        RPCA_CHECK_LAUNCH();
        if (max_chunks > 0) {
            if (vec && lp <= 64) {
                spmm_heavy_group_kernel<8><<<grid_for(max_chunks * 8, 256), 256, 0, s>>>(
                    ptr, idx, val, first, rows, cols, nnz, table, max_chunks, X, lp, part);
            } else if (vec && lp <= 128) {
                spmm_heavy_group_kernel<16><<<grid_for(max_chunks * 16, 256), 256, 0, s>>>(
                    ptr, idx, val, first, rows, cols, nnz, table, max_chunks, X, lp, part);
            } else if (vec && lp <= 256) {
                spmm_heavy_group_kernel<32><<<grid_for(max_chunks * 32, 256), 256, 0, s>>>(
                    ptr, idx, val, first, rows, cols, nnz, table, max_chunks, X, lp, part);
            } else {
                spmm_heavy_kernel<<<grid_for(max_chunks * 32, 256), 256, 0, s>>>(ptr, idx, val, first, rows, cols,
                                                                                nnz, table, max_chunks, X, lp, part);
            }
            RPCA_CHECK_LAUNCH();
            spmm_heavy_reduce_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(max_chunks, (int64_t)num_sms() * 8)),
                                       kReduceWarps * 32, 0, s>>>(first, table, rows, max_chunks, part, lp, Y);
            RPCA_CHECK_LAUNCH();
        }
        return RPCA_OK;
    }
};

int64_t max_chunks_for(int64_t nnz, int64_t rows) {
    // sum over heavy rows (deg > kHeavy) of ceil(deg / kHeavy) < 2 nnz / kHeavy
    (void)rows;
    return 2 * (nnz / kHeavy) + 1;
}

struct CsrScratch {
    size_t row_of = 0, keys0 = 0, keys1 = 0, rows0 = 0, rows1 = 0, vals0 = 0, vals1 = 0, hist = 0, tptr = 0,
           first_a = 0, first_t = 0, table_a = 0, table_t = 0, part_a = 0, part_t = 0, scan = 0, perm_a = 0,
           perm_t = 0, bk_a = 0, bk_t = 0, total = 0;
};

CsrScratch csr_scratch(int64_t m, int64_t n, int64_t nnz, int max_lp) {
    CsrScratch S;
    size_t off = 0;
    auto take = [&](size_t b) { const size_t o = off; off = (off + b + 255) & ~(size_t)255; return o; };
    const int64_t nblocks = cdiv(std::max<int64_t>(nnz, 1), kTile);
    S.row_of = take((size_t)nnz * 4);
    S.keys0 = take((size_t)nnz * 4);
    S.keys1 = take((size_t)nnz * 4);
    S.rows0 = take((size_t)nnz * 4);
    S.rows1 = take((size_t)nnz * 4);
    S.vals0 = take((size_t)nnz * 4);
    S.vals1 = take((size_t)nnz * 4);
    S.hist = take((size_t)256 * nblocks * 4);
    S.tptr = take((size_t)(n + 1) * 4);
    S.first_a = take((size_t)(m + 1) * 4);
    S.first_t = take((size_t)(n + 1) * 4);
    S.table_a = take((size_t)max_chunks_for(nnz, m) * 8);
    S.table_t = take((size_t)max_chunks_for(nnz, n) * 8);
    S.part_a = take((size_t)max_chunks_for(nnz, m) * max_lp * 4);
    S.part_t = take((size_t)max_chunks_for(nnz, n) * max_lp * 4);
    S.scan = take((size_t)scan_tiles(std::max({(int64_t)256 * nblocks, m + 1, n + 1})) * 8);
    S.perm_a = take((size_t)m * 4);
    S.perm_t = take((size_t)n * 4);
    S.bk_a = take((size_t)(2 * kBuckets + 1) * 4);
    S.bk_t = take((size_t)(2 * kBuckets + 1) * 4);
    S.total = off;
    return S;
}

// A (CSR) and A^T (CSR, built by the stable sort) as the pipeline's operator.
struct CsrOp final : Operator {
    Spmm a, t;
    int apply(const float *X, int lp, float *Y, cudaStream_t s, const float *) const override {
        TimedScope ts(kTimeApplyKernel, s);
        return a.run(X, lp, Y, s);
    }
    int adjoint_splits(int) const override { return 1; }
    int adjoint(const float *Q, int lp, float *part, cudaStream_t s) const override {
        TimedScope ts(kTimeAdjointKernel, s);
        return t.run(Q, lp, part, s);
    }
};

// Build A^T from A and the SpMM plans of both, inside the scratch at `base`.
int prepare(CsrOp &op, const int32_t *row_ptr, const int32_t *col_idx, const float *val, int64_t m, int64_t n,
            int64_t nnz, char *base, const CsrScratch &S, DevStatus *st, cudaStream_t s) {
    auto I = [&](size_t o) { return reinterpret_cast<int32_t *>(base + o); };
    auto F = [&](size_t o) { return reinterpret_cast<float *>(base + o); };
    op.m = m; op.n = n;
    op.a.ptr = row_ptr; op.a.idx = col_idx; op.a.val = val;
    op.a.rows = m; op.a.cols = n; op.a.nnz = nnz; op.a.max_chunks = max_chunks_for(nnz, m);
    op.a.first = I(S.first_a); op.a.table = reinterpret_cast<int2 *>(base + S.table_a); op.a.part = F(S.part_a);
    op.a.scan_tmp = reinterpret_cast<int64_t *>(base + S.scan);
    op.a.perm = I(S.perm_a); op.a.bk = I(S.bk_a);

    int32_t *keys[2] = {I(S.keys0), I(S.keys1)};
    int32_t *rws[2] = {I(S.rows0), I(S.rows1)};
    float *vls[2] = {F(S.vals0), F(S.vals1)};
    int cur = 0;
    csr_check_kernel<<<grid_for(std::max(m, nnz), 256), 256, 0, s>>>(row_ptr, col_idx, m, n, nnz, st);
    RPCA_CHECK_LAUNCH();
    if (nnz > 0) {
        if (cudaMemsetAsync(rws[0], 0, (size_t)nnz * sizeof(int32_t), s) != cudaSuccess) return RPCA_ERR_CUDA;
        row_expand_kernel<<<grid_for(m * 32, 256), 256, 0, s>>>(row_ptr, m, nnz, rws[0]);
        RPCA_CHECK_LAUNCH();
        copy_i32_kernel<<<grid_for(nnz, 256), 256, 0, s>>>(col_idx, keys[0], nnz);
        RPCA_CHECK_LAUNCH();
        copy_f32_kernel<<<grid_for(nnz, 256), 256, 0, s>>>(val, vls[0], nnz);
        RPCA_CHECK_LAUNCH();
        const int nblocks = (int)cdiv(nnz, kTile);
        int bits = 1;
        while (bits < 31 && (1LL << bits) < n) ++bits;
        for (int shift = 0; shift < bits; shift += 8) {
            radix_hist_kernel<<<nblocks, kSortThreads, 0, s>>>(keys[cur], nnz, shift, I(S.hist), nblocks);
            RPCA_CHECK_LAUNCH();
            RPCA_TRY(launch_scan(I(S.hist), (int64_t)256 * nblocks, reinterpret_cast<int64_t *>(base + S.scan), s));
            radix_scatter_kernel<<<nblocks, kSortThreads, 0, s>>>(keys[cur], rws[cur], vls[cur], nnz, shift, I(S.hist),
                                                                 nblocks, keys[cur ^ 1], rws[cur ^ 1], vls[cur ^ 1]);
            RPCA_CHECK_LAUNCH();
            cur ^= 1;
        }
    }
    colptr_kernel<<<grid_for(n + 1, 256), 256, 0, s>>>(keys[cur], nnz, n, I(S.tptr));
    RPCA_CHECK_LAUNCH();
    op.t.ptr = I(S.tptr); op.t.idx = rws[cur]; op.t.val = vls[cur];
    op.t.rows = n; op.t.cols = m; op.t.nnz = nnz; op.t.max_chunks = max_chunks_for(nnz, n);
    op.t.first = I(S.first_t); op.t.table = reinterpret_cast<int2 *>(base + S.table_t); op.t.part = F(S.part_t);
    op.t.scan_tmp = reinterpret_cast<int64_t *>(base + S.scan);
    op.t.perm = I(S.perm_t); op.t.bk = I(S.bk_t);
    RPCA_TRY(op.a.plan(s));
    RPCA_TRY(op.t.plan(s));
    return RPCA_OK;
}

bool csr_args_ok(int64_t m, int64_t n, int64_t nnz, const int32_t *row_ptr, const int32_t *col_idx, const float *val) {
    if (m < 1 || n < 1 || nnz < 0 || nnz > INT32_MAX || m >= INT32_MAX || n >= INT32_MAX || !row_ptr) return false;
    if (nnz > 0 && (!col_idx || !val)) return false;
    return true;
}

}  // namespace

}  // namespace rpca

extern "C" size_t rpca_csr_workspace_size(int64_t m, int64_t n, int64_t nnz, const rpca_opts *o) {
    if (!o || m < 1 || n < 1 || nnz < 0 || o->l < 1 || o->k < 1 || o->l > RPCA_MAX_L) return 0;
    const int lp = rpca::padded_l(o->l);
    const rpca::CsrScratch S = rpca::csr_scratch(m, n, nnz, lp);
    return rpca::make_layout(m, n, o->l, o->k, 1, S.total).total;
}

extern "C" int rpca_csr(int64_t m, int64_t n, int64_t nnz, const int32_t *row_ptr, const int32_t *col_idx,
                        const float *val, const rpca_opts *o, float *U, int64_t ldu, float *S, float *V,
                        int64_t ldv, void *ws, size_t ws_bytes, rpca_stream_t stream) {
    if (!o || !rpca::csr_args_ok(m, n, nnz, row_ptr, col_idx, val)) return RPCA_ERR_INVALID_ARG;
    const size_t need = rpca_csr_workspace_size(m, n, nnz, o);
    RPCA_TRY(rpca::check_common(m, n, o, U, ldu, S, V, ldv, ws, ws_bytes, need));
    if (rpca::renorm_kind(o->renorm) == RPCA_RENORM_LU && !rpca::tslu_supported(o->l)) return RPCA_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    const int lp = rpca::padded_l(o->l);
    const rpca::CsrScratch SC = rpca::csr_scratch(m, n, nnz, lp);
    const rpca::Layout L = rpca::make_layout(m, n, o->l, o->k, 1, SC.total);
    rpca::CsrOp op;
    auto *st = reinterpret_cast<rpca::DevStatus *>(reinterpret_cast<char *>(ws) + L.status);
    if (cudaMemsetAsync(st, 0, sizeof(rpca::DevStatus), s) != cudaSuccess) return RPCA_ERR_CUDA;
    RPCA_TRY(rpca::prepare(op, row_ptr, col_idx, val, m, n, nnz, reinterpret_cast<char *>(ws) + L.scratch, SC, st, s));
    return rpca::run_pipeline(op, o, U, ldu, S, V, ldv, ws, L, s, /*clear_status=*/false);
}

extern "C" size_t rpca_resid_csr_workspace_size(int64_t m, int64_t n, int64_t nnz, int32_t k) {
    if (m < 1 || n < 1 || nnz < 0 || k < 0 || k > RPCA_MAX_L) return 0;
    const rpca::CsrScratch S = rpca::csr_scratch(m, n, nnz, 8);
    const rpca::ResidLayout R = rpca::make_resid_layout(m, n, k, 1);
    return ((R.total + 255) & ~(size_t)255) + S.total;
}

extern "C" int rpca_resid_norm_csr(int64_t m, int64_t n, int64_t nnz, const int32_t *row_ptr, const int32_t *col_idx,
                                   const float *val, int32_t raw, const float *U, int64_t ldu, const float *S,
                                   const float *V, int64_t ldv, int32_t k, int32_t iters, uint64_t seed, double *est,
                                   void *ws, size_t ws_bytes, rpca_stream_t stream) {
    if (!rpca::csr_args_ok(m, n, nnz, row_ptr, col_idx, val) || !est || k < 0 || k > RPCA_MAX_L || iters < 1)
        return RPCA_ERR_INVALID_ARG;
    if (k > 0 && (!U || !S || !V || ldu < k || ldv < k)) return RPCA_ERR_INVALID_ARG;
    const size_t need = rpca_resid_csr_workspace_size(m, n, nnz, k);
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0 || ws_bytes < need) return RPCA_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    const rpca::ResidLayout R = rpca::make_resid_layout(m, n, k, 1);
    const rpca::CsrScratch SC = rpca::csr_scratch(m, n, nnz, 8);
    rpca::CsrOp op;
    char *base = reinterpret_cast<char *>(ws) + ((R.total + 255) & ~(size_t)255);
    auto *st = reinterpret_cast<rpca::DevStatus *>(reinterpret_cast<char *>(ws) + R.status);
    if (cudaMemsetAsync(st, 0, sizeof(rpca::DevStatus), s) != cudaSuccess) return RPCA_ERR_CUDA;
    RPCA_TRY(rpca::prepare(op, row_ptr, col_idx, val, m, n, nnz, base, SC, st, s));
    return rpca::run_resid(op, raw, U, ldu, S, V, ldv, k, iters, seed, est, ws, R, s, /*clear_status=*/false);
}

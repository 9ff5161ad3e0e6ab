// Sparse A in CSR form.  Section 5 notes that the same code serves dense and
// sparse A: only the two products change.  A X is a gather SpMM over the rows
// of A; A^T Q is the same SpMM over the rows of A^T, which is built once per
// call by a stable radix sort of the nonzeros by column (no atomics anywhere,
// so every result is deterministic).
//
// SpMM: one warp per row, lanes across the l-wide block (the block operand is
// read from L2 row by row), eight nonzeros per step so that eight gathers are
// in flight per warp.  Rows with more than kHeavy nonzeros (power-law degree
// distributions have rows with ~1e5 of them) are cut into chunks of kHeavy
// nonzeros, one warp per chunk writing a partial row, and a third kernel adds
// each heavy row's partials in chunk order.
#include "pipeline.cuh"
#include "resid.cuh"

namespace rpca {

namespace {

constexpr int kHeavy = 256;
constexpr int kTile = 4096;            // radix sort: nonzeros per block (8 warps x 512)
constexpr int kSortThreads = 256;

__device__ __forceinline__ int64_t upper_bound_ptr(const int32_t *__restrict__ ptr, int64_t rows, int64_t p) {
    // largest r in [0, rows) with ptr[r] <= p
    int64_t lo = 0, hi = rows;                 // invariant: ptr[lo] <= p, answer in [lo, hi)
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if ((int64_t)ptr[mid] <= p) lo = mid; else hi = mid;
    }
    return lo;
}

__global__ void nnz_row_kernel(const int32_t *__restrict__ ptr, int64_t rows, int64_t nnz, int32_t *__restrict__ row_of) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x)
        row_of[p] = (int32_t)upper_bound_ptr(ptr, rows, p);
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

// in-place exclusive scan of `total` counts, one CTA
__global__ void __launch_bounds__(1024) scan_kernel(int32_t *__restrict__ data, int64_t total) {
    __shared__ int64_t sums[1024];
    const int64_t per = (total + blockDim.x - 1) / blockDim.x;
    const int64_t b = threadIdx.x * per, e = min(total, b + per);
    int64_t s = 0;
    for (int64_t i = b; i < e; ++i) s += data[i];
    sums[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t run = 0;
        for (int t = 0; t < (int)blockDim.x; ++t) { const int64_t v = sums[t]; sums[t] = run; run += v; }
    }
    __syncthreads();
    int64_t run = sums[threadIdx.x];
    for (int64_t i = b; i < e; ++i) { const int32_t v = data[i]; data[i] = (int32_t)run; run += v; }
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

// heavy rows: Y[r] = sum of its chunk partials in chunk order
__global__ void __launch_bounds__(256)
spmm_heavy_reduce_kernel(const int32_t *__restrict__ first, int64_t rows, int64_t max_chunks,
                         const float *__restrict__ part, int lp, float *__restrict__ Y) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = wid; r < rows; r += nw) {
        const int64_t c0 = first[r], c1 = min((int64_t)first[r + 1], max_chunks);
        if (c1 <= c0) continue;
        for (int c = lane; c < lp; c += 32) {
            float s = 0.f;
            for (int64_t ch = c0; ch < c1; ++ch) s += part[ch * lp + c];
            Y[r * lp + c] = s;
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
    int2 *table = nullptr;         // max_chunks
    float *part = nullptr;         // max_chunks x max_lp

    int plan(cudaStream_t s) const {
        chunk_count_kernel<<<grid_for(rows + 1, 256), 256, 0, s>>>(ptr, rows, first);
        RPCA_CHECK_LAUNCH();
        scan_kernel<<<1, 1024, 0, s>>>(first, rows + 1);
        RPCA_CHECK_LAUNCH();
        if (max_chunks > 0) {
            chunk_table_kernel<<<grid_for(rows, 256), 256, 0, s>>>(ptr, first, rows, table, max_chunks);
            RPCA_CHECK_LAUNCH();
        }
        return RPCA_OK;
    }
    int run(const float *X, int lp, float *Y, cudaStream_t s) const {
        spmm_light_kernel<<<grid_for(rows * 32, 256), 256, 0, s>>>(ptr, idx, val, rows, cols, nnz, X, lp, Y);
        RPCA_CHECK_LAUNCH();
        if (max_chunks > 0) {
            spmm_heavy_kernel<<<grid_for(max_chunks * 32, 256), 256, 0, s>>>(ptr, idx, val, first, rows, cols, nnz,
                                                                            table, max_chunks, X, lp, part);
            RPCA_CHECK_LAUNCH();
            spmm_heavy_reduce_kernel<<<grid_for(rows * 32, 256), 256, 0, s>>>(first, rows, max_chunks, part, lp, Y);
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
           first_a = 0, first_t = 0, table_a = 0, table_t = 0, part_a = 0, part_t = 0, total = 0;
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
    S.total = off;
    return S;
}

// A (CSR) and A^T (CSR, built by the stable sort) as the pipeline's operator.
struct CsrOp final : Operator {
    Spmm a, t;
    int apply(const float *X, int lp, float *Y, cudaStream_t s) const override { return a.run(X, lp, Y, s); }
    int adjoint_splits(int) const override { return 1; }
    int adjoint(const float *Q, int lp, float *part, cudaStream_t s) const override { return t.run(Q, lp, part, s); }
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

    int32_t *keys[2] = {I(S.keys0), I(S.keys1)};
    int32_t *rws[2] = {I(S.rows0), I(S.rows1)};
    float *vls[2] = {F(S.vals0), F(S.vals1)};
    int cur = 0;
    csr_check_kernel<<<grid_for(std::max(m, nnz), 256), 256, 0, s>>>(row_ptr, col_idx, m, n, nnz, st);
    RPCA_CHECK_LAUNCH();
    if (nnz > 0) {
        nnz_row_kernel<<<grid_for(nnz, 256), 256, 0, s>>>(row_ptr, m, nnz, rws[0]);
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
            scan_kernel<<<1, 1024, 0, s>>>(I(S.hist), (int64_t)256 * nblocks);
            RPCA_CHECK_LAUNCH();
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
    if (o->renorm != RPCA_RENORM_CHOLQR) return RPCA_ERR_UNSUPPORTED;
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

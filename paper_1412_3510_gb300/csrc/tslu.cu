// Tall-skinny LU with tournament pivoting: the LU renormalisation of Section 5
// (every product but the last is renormalised by an LU factorisation with
// partial pivoting, Q <- P^T L = Y U^-1) for tall Y on the GPU.
//
// Partial pivoting on an m x l block picks its l pivot rows one column at a time
// across all m rows; the tournament (Grigori, Demmel & Xiang, SIAM J. Matrix Anal.
// Appl. 32 (2011)) picks them in a tree instead: every node runs partial-pivoting
// LU on at most 2l rows and passes its l pivot rows up; level 0 takes blocks of 2l
// consecutive rows of Y, each later level merges pairs of candidate sets.  The l
// rows that win are factored (W = P L U, partial pivoting), and the renormalised
// block is Y U^-1, as with the exact LU (Y = P^T L U gives P^T L = Y U^-1).  Only
// the span of the block enters the next product, so any such U serves.
#include "internal.cuh"
#include "gepp.cuh"

namespace rpca {

namespace {

constexpr int kLuThreads = 512;

// One tournament node: partial-pivoting elimination of the rows cand[base ..
// base + per_node) (row indices of Y; cand == nullptr: the rows themselves; entries
// past ncand or < 0 are absent) on the first l columns; out[node * l + j] = the row of
// Y chosen as pivot j (-1 when the node has fewer than j + 1 rows).
__global__ void __launch_bounds__(kLuThreads) tslu_node_kernel(const float *__restrict__ Y, int64_t rows, int lp,
                                                               int l, const int32_t *__restrict__ cand,
                                                               int64_t ncand, int per_node,
                                                               int32_t *__restrict__ out) {
    extern __shared__ float sm[];
    const int ld = l + 1;
    float *M = sm;                                        // per_node x ld
    int *ids = reinterpret_cast<int *>(sm + (size_t)per_node * ld);
    __shared__ GeppScratch g;
    const int tid = threadIdx.x;
    const int64_t base = (int64_t)blockIdx.x * per_node;
    for (int r = tid; r < per_node; r += kLuThreads) {
        const int64_t pos = base + r;
        int id = -1;
        if (pos < ncand) id = cand ? cand[pos] : (int)pos;
        if (id >= rows) id = -1;
        ids[r] = id;
    }
    __syncthreads();
    for (int e = tid; e < per_node * l; e += kLuThreads) {
        const int r = e / l, c = e - r * l;
        const int id = ids[r];
        M[r * ld + c] = id >= 0 ? Y[(int64_t)id * lp + c] : 0.f;
    }
    __syncthreads();
    const int j = gepp_block(M, ld, ids, per_node, l, g);
    for (int t = tid; t < l; t += kLuThreads) out[(int64_t)blockIdx.x * l + t] = t < j ? ids[t] : -1;
}

}  // namespace

size_t tslu_ids_bytes(int64_t rows, int l) {
    return ((size_t)cdiv(std::max<int64_t>(rows, 1), (int64_t)2 * l) * l + l) * sizeof(int32_t);
}

bool tslu_supported(int l) { return l >= 1 && l <= 160; }

// The l pivot rows of Y (rows x lp, first l columns) by the tournament; *winner
// points to them (in buf0 or buf1, each tslu_ids_bytes(rows, l) bytes).
int launch_tslu_select(const float *Y, int64_t rows, int lp, int l, int32_t *buf0, int32_t *buf1,
                       const int32_t **winner, cudaStream_t s) {
    if (!tslu_supported(l) || rows > INT32_MAX) return RPCA_ERR_UNSUPPORTED;   // row ids are int32
    const int per = 2 * l;
    const size_t smem = (size_t)per * (l + 1) * sizeof(float) + (size_t)per * sizeof(int);
    if (cudaFuncSetAttribute(tslu_node_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return RPCA_ERR_CUDA;
    int64_t nodes = cdiv(rows, (int64_t)per);
    tslu_node_kernel<<<(unsigned)nodes, kLuThreads, smem, s>>>(Y, rows, lp, l, nullptr, rows, per, buf0);
    RPCA_CHECK_LAUNCH();
    int32_t *cur = buf0, *nxt = buf1;
    while (nodes > 1) {
        const int64_t ncand = nodes * l;
        nodes = cdiv(ncand, (int64_t)per);
        tslu_node_kernel<<<(unsigned)nodes, kLuThreads, smem, s>>>(Y, rows, lp, l, cur, ncand, per, nxt);
        RPCA_CHECK_LAUNCH();
        std::swap(cur, nxt);
    }
    *winner = cur;
    return RPCA_OK;
}

}  // namespace rpca

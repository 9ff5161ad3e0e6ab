// Plain FP32 (FFMA) tall-skinny products: the "plain FP32 GPU form" of every
// product of the method (Section 2's A*Omega and the power iterations'
// alternating A and A^* applications, Section 5's (Q'*A)' adjoint, the Gram
// matrices of the renormalisations and the lifts U = Q W of Eq. i4).
//
// C = op(A) * B with op(A) = A (row-major M x K) or A^T (A stored K x M, so
// that A^T Y streams A row by row exactly like A X does).  The K range can be
// split over grid.z; slice z writes its own partial C + z * split_stride and a
// separate kernel reduces the slices in a fixed order (deterministic).
//
// Register-blocked SIMT: 256 threads, CTA tile BM x BN, K step BK, each thread
// a TM x TN micro-tile; tiles staged in shared memory with a register prefetch
// of the next K step (the global loads of step t+1 are in flight while step t
// computes).
#include "internal.cuh"

#include <algorithm>

namespace rpca {

namespace {

constexpr int kThreads = 256;
constexpr int kBK = 32;

__device__ __forceinline__ bool aligned16(const void *p) {
    return (reinterpret_cast<uintptr_t>(p) & 15u) == 0;
}

template <int BM, int BN, int TM, int TN, bool TRANS_A>
__global__ void __launch_bounds__(kThreads)
sgemm_kernel(int64_t M, int64_t N, int64_t K, const float *__restrict__ A, int64_t lda,
             const float *__restrict__ B, int64_t ldb, float *__restrict__ C, int64_t ldc,
             int64_t kchunk, int64_t split_stride, const int *__restrict__ copy_flag,
             const float *__restrict__ bias) {
    constexpr int BK = kBK;
    constexpr int TX = BN / TN;
    constexpr int TY = BM / TM;
    static_assert(TX * TY == kThreads, "thread grid must cover the tile");
    constexpr int APAD = 4, BPAD = 4;
    // A tile as As[k][m] (m contiguous), B tile as Bs[k][n].
    __shared__ __align__(16) float As[BK][BM + APAD];
    __shared__ __align__(16) float Bs[BK][BN + BPAD];

    constexpr int A_F4 = BM * BK / 4 / kThreads;                 // float4 slots per thread
    constexpr int B_F4 = (BN * BK / 4 + kThreads - 1) / kThreads;
    static_assert(A_F4 >= 1, "A tile too small");

    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int64_t m0 = (int64_t)blockIdx.x * BM;
    const int64_t n0 = (int64_t)blockIdx.y * BN;
    if (!TRANS_A && copy_flag && *copy_flag == 0) {
        // multiplication by the identity: C = A on this tile
        if (blockIdx.z == 0)
            for (int e = tid; e < BM * BN; e += kThreads) {
                const int64_t r = m0 + e / BN, c = n0 + e % BN;
                if (r < M && c < N) C[r * ldc + c] = A[r * lda + c];
            }
        return;
    }
    const int64_t kbeg = (int64_t)blockIdx.z * kchunk;
    const int64_t kend = min(K, kbeg + kchunk);
    C += (int64_t)blockIdx.z * split_stride;
    if (kbeg >= kend) {
        // empty slice: still define the partial
        for (int i = 0; i < TM; ++i)
            for (int j = 0; j < TN; ++j) {
                const int64_t r = m0 + ty * TM + i, c = n0 + tx * TN + j;
                if (r < M && c < N) C[r * ldc + c] = 0.f;
            }
        return;
    }

    const bool vecA = aligned16(A) && (lda % 4 == 0);
    const bool vecB = aligned16(B) && (ldb % 4 == 0);

    float ra[A_F4][4];
    float rb[B_F4][4];

    auto load_tiles = [&](int64_t k0) {
#pragma unroll
        for (int q = 0; q < A_F4; ++q) {
            const int f = tid + q * kThreads;
            int64_t row, col;              // element (row, col) of the stored A
            int64_t rbound, cbound;
            if (!TRANS_A) {                // stored M x K: rows = m, 4 consecutive k
                const int r = f / (BK / 4), kq = f % (BK / 4);
                row = m0 + r; col = k0 + 4 * kq; rbound = M; cbound = kend;
            } else {                       // stored K x M: rows = k, 4 consecutive m
                const int kr = f / (BM / 4), mq = f % (BM / 4);
                row = k0 + kr; col = m0 + 4 * mq; rbound = kend; cbound = M;
            }
            const float *p = A + row * lda + col;
            if (row < rbound && col + 3 < cbound && vecA) {
                const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
                ra[q][0] = v.x; ra[q][1] = v.y; ra[q][2] = v.z; ra[q][3] = v.w;
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    ra[q][e] = (row < rbound && col + e < cbound) ? __ldg(p + e) : 0.f;
            }
        }
#pragma unroll
        for (int q = 0; q < B_F4; ++q) {
            const int f = tid + q * kThreads;
            if (f < BN * BK / 4) {
                const int kr = f / (BN / 4), nq = f % (BN / 4);
                const int64_t row = k0 + kr, col = n0 + 4 * nq;
                const float *p = B + row * ldb + col;
                if (row < kend && col + 3 < N && vecB) {
                    const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
                    rb[q][0] = v.x; rb[q][1] = v.y; rb[q][2] = v.z; rb[q][3] = v.w;
                } else {
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        rb[q][e] = (row < kend && col + e < N) ? __ldg(p + e) : 0.f;
                }
            }
        }
    };

    auto store_tiles = [&]() {
#pragma unroll
        for (int q = 0; q < A_F4; ++q) {
            const int f = tid + q * kThreads;
            if (!TRANS_A) {
                const int r = f / (BK / 4), kq = f % (BK / 4);
#pragma unroll
                for (int e = 0; e < 4; ++e) As[4 * kq + e][r] = ra[q][e];
            } else {
                const int kr = f / (BM / 4), mq = f % (BM / 4);
                *reinterpret_cast<float4 *>(&As[kr][4 * mq]) =
                    make_float4(ra[q][0], ra[q][1], ra[q][2], ra[q][3]);
            }
        }
#pragma unroll
        for (int q = 0; q < B_F4; ++q) {
            const int f = tid + q * kThreads;
            if (f < BN * BK / 4) {
                const int kr = f / (BN / 4), nq = f % (BN / 4);
                *reinterpret_cast<float4 *>(&Bs[kr][4 * nq]) =
                    make_float4(rb[q][0], rb[q][1], rb[q][2], rb[q][3]);
            }
        }
    };

    float acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;

    const int64_t ntiles = (kend - kbeg + BK - 1) / BK;
    load_tiles(kbeg);
    store_tiles();
    __syncthreads();
    for (int64_t t = 0; t < ntiles; ++t) {
        if (t + 1 < ntiles) load_tiles(kbeg + (t + 1) * BK);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float a[TM], b[TN];
#pragma unroll
            for (int i = 0; i < TM; i += 4) {
                const float4 v = *reinterpret_cast<const float4 *>(&As[kk][ty * TM + i]);
                a[i] = v.x; a[i + 1] = v.y; a[i + 2] = v.z; a[i + 3] = v.w;
            }
            if constexpr (TN % 4 == 0) {
#pragma unroll
                for (int j = 0; j < TN; j += 4) {
                    const float4 v = *reinterpret_cast<const float4 *>(&Bs[kk][tx * TN + j]);
                    b[j] = v.x; b[j + 1] = v.y; b[j + 2] = v.z; b[j + 3] = v.w;
                }
            } else {
#pragma unroll
                for (int j = 0; j < TN; j += 2) {
                    const float2 v = *reinterpret_cast<const float2 *>(&Bs[kk][tx * TN + j]);
                    b[j] = v.x; b[j + 1] = v.y;
                }
            }
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
        if (t + 1 < ntiles) {
            store_tiles();
            __syncthreads();
        }
    }

    if (!TRANS_A && bias) {
        // implicit centring (Section 5): C = A B - 1 (c B), the row vector c B given
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int64_t c = n0 + tx * TN + j;
            const float bj = c < N ? bias[c] : 0.f;
#pragma unroll
            for (int i = 0; i < TM; ++i) acc[i][j] -= bj;
        }
    }
    const bool vecC = aligned16(C) && (ldc % 4 == 0) && (TN % 4 == 0);
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int64_t r = m0 + ty * TM + i;
        if (r >= M) continue;
        float *crow = C + r * ldc;
#pragma unroll
        for (int j = 0; j < TN; j += 4) {
            const int64_t c = n0 + tx * TN + j;
            if (TN % 4 == 0 && vecC && c + 3 < N) {
                *reinterpret_cast<float4 *>(crow + c) =
                    make_float4(acc[i][j], acc[i][j + 1], acc[i][j + 2], acc[i][j + 3]);
            } else {
#pragma unroll
                for (int e = 0; e < 4 && j + e < TN; ++e)
                    if (c + e < N) crow[c + e] = acc[i][j + e];
            }
        }
    }
}

template <int BM, int BN, int TM, int TN>
int launch_cfg(bool trans_a, int64_t M, int64_t N, int64_t K, const float *A, int64_t lda,
               const float *B, int64_t ldb, float *C, int64_t ldc, int splits,
               int64_t split_stride, cudaStream_t s, const int *copy_flag, const float *bias) {
    const int64_t kchunk = round_up(cdiv(K, splits), kBK);
    const int64_t gz = cdiv(K, kchunk);
    // slices past the end of K still write zero partials so the reduction sees `splits` slices
    dim3 grid((unsigned)cdiv(M, BM), (unsigned)cdiv(N, BN), (unsigned)std::max<int64_t>(splits, gz));
    if (grid.x == 0 || grid.y == 0) return RPCA_OK;
    if (grid.x > 2147483647u || grid.y > 65535u || grid.z > 65535u) return RPCA_ERR_INVALID_ARG;
    if (trans_a)
        sgemm_kernel<BM, BN, TM, TN, true><<<grid, kThreads, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc,
                                                                     kchunk, split_stride, nullptr, nullptr);
    else
        sgemm_kernel<BM, BN, TM, TN, false><<<grid, kThreads, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc,
                                                                      kchunk, split_stride, copy_flag, bias);
    RPCA_CHECK_LAUNCH();
    return RPCA_OK;
}

}  // namespace

int choose_splits(int64_t M, int64_t N, int64_t K) {
    const int64_t bn = N <= 16 ? 16 : N <= 32 ? 32 : N <= 64 ? 64 : 128;
    const int64_t tiles = cdiv(M, 128) * cdiv(N, bn);
    const int64_t want = 2LL * num_sms();
    int64_t s = cdiv(want, tiles);
    s = std::min<int64_t>(s, std::max<int64_t>(1, K / (4 * kBK)));
    return (int)std::max<int64_t>(1, std::min<int64_t>(s, 4096));
}

// C (M x N) = A (M x K) B (K x N) for the small right-hand factors of the
// pipeline (Y R^-1 with K = N = lp, the lifts Q W and Q2 Z with N = k): B whole in
// shared memory, a 16 RPT-row tile of A, a 16 x 16 thread grid where thread (ty, tx)
// owns rows ty + 16 i (i < RPT) and columns tx + 16 j (j < NG).  RPT = 1 for short
// blocks (the n side: a few thousand rows spread over many SMs), 4 for long ones.
// copy_flag == 0 makes B the identity (C = A, N == K).
template <int NG, int RPT>
__global__ void __launch_bounds__(256) smallk_gemm_kernel(int64_t M, int N, int K, const float *__restrict__ A,
                                                          int64_t lda, const float *__restrict__ B, int64_t ldb,
                                                          float *__restrict__ C, int64_t ldc,
                                                          const int *__restrict__ copy_flag,
                                                          const float *__restrict__ bias) {
    extern __shared__ float sk[];
    constexpr int NB = 16 * NG;                  // B columns in shared memory
    constexpr int kRows = 16 * RPT;              // rows of A per CTA
    const int lda_s = K + 1;                     // odd: the 16 row-owners hit 16 banks
    float *Bs = sk;                              // K x NB
    float *As = sk + (size_t)K * NB;             // kRows x lda_s
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t m0 = (int64_t)blockIdx.x * kRows;
    if (copy_flag && *copy_flag == 0) {
        for (int e = tid; e < kRows * N; e += 256) {
            const int64_t r = m0 + e / N;
            const int c = e % N;
            if (r < M) C[r * ldc + c] = A[r * lda + c];
        }
        return;
    }
    for (int e = tid; e < K * NB; e += 256) {
        const int k = e / NB, c = e - k * NB;
        Bs[e] = c < N ? B[(int64_t)k * ldb + c] : 0.f;
    }
    for (int e = tid; e < kRows * K; e += 256) {
        const int r = e / K, k = e - r * K;
        As[r * lda_s + k] = m0 + r < M ? A[(m0 + r) * lda + k] : 0.f;
    }
    __syncthreads();
    float acc[RPT][NG];
#pragma unroll
    for (int i = 0; i < RPT; ++i)
#pragma unroll
        for (int j = 0; j < NG; ++j) acc[i][j] = 0.f;
    for (int k = 0; k < K; ++k) {
        float a[RPT], b[NG];
#pragma unroll
        for (int i = 0; i < RPT; ++i) a[i] = As[(ty + 16 * i) * lda_s + k];
#pragma unroll
        for (int j = 0; j < NG; ++j) b[j] = Bs[k * NB + tx + 16 * j];
#pragma unroll
        for (int i = 0; i < RPT; ++i)
#pragma unroll
            for (int j = 0; j < NG; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
        const int64_t r = m0 + ty + 16 * i;
        if (r >= M) continue;
#pragma unroll
        for (int j = 0; j < NG; ++j) {
            const int c = tx + 16 * j;
            if (c < N) C[r * ldc + c] = bias ? acc[i][j] - bias[c] : acc[i][j];
        }
    }
}

template <int NG>
int launch_smallk(int64_t M, int N, int K, const float *A, int64_t lda, const float *B, int64_t ldb, float *C,
                  int64_t ldc, cudaStream_t s, const int *copy_flag, const float *bias) {
    // 64-row tiles while they fill two waves of the SMs, 16-row tiles below that
    const bool short_block = cdiv(M, (int64_t)64) < 2LL * num_sms();
    const int rows = short_block ? 16 : 64;
    const size_t smem = ((size_t)K * 16 * NG + (size_t)rows * (K + 1)) * sizeof(float);
    auto kern = short_block ? smallk_gemm_kernel<NG, 1> : smallk_gemm_kernel<NG, 4>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return RPCA_ERR_CUDA;
    kern<<<(unsigned)cdiv(M, (int64_t)rows), 256, smem, s>>>(M, N, K, A, lda, B, ldb, C, ldc, copy_flag, bias);
    RPCA_CHECK_LAUNCH();
    return RPCA_OK;
}

int launch_sgemm(bool trans_a, int64_t M, int64_t N, int64_t K, const float *A, int64_t lda,
                 const float *B, int64_t ldb, float *C, int64_t ldc, int splits,
                 int64_t split_stride, cudaStream_t s, const int *copy_flag, const float *bias) {
    if (M <= 0 || N <= 0) return RPCA_OK;
    if (bias && (trans_a || splits > 1)) return RPCA_ERR_INVALID_ARG;
    if (splits < 1) splits = 1;
    if (!trans_a && splits == 1 && K >= 1 && K <= 160 && N <= 160 && (!copy_flag || N == K)) {
        const int ng = (int)cdiv(N, (int64_t)16), n = (int)N, k = (int)K;
        switch (ng) {
            case 1: return launch_smallk<1>(M, n, k, A, lda, B, ldb, C, ldc, s, copy_flag, bias);
            case 2: return launch_smallk<2>(M, n, k, A, lda, B, ldb, C, ldc, s, copy_flag, bias);
            case 3: return launch_smallk<3>(M, n, k, A, lda, B, ldb, C, ldc, s, copy_flag, bias);
            case 4: return launch_smallk<4>(M, n, k, A, lda, B, ldb, C, ldc, s, copy_flag, bias);
            case 5: return launch_smallk<5>(M, n, k, A, lda, B, ldb, C, ldc, s, copy_flag, bias);
            case 6: return launch_smallk<6>(M, n, k, A, lda, B, ldb, C, ldc, s, copy_flag, bias);
            case 7: return launch_smallk<7>(M, n, k, A, lda, B, ldb, C, ldc, s, copy_flag, bias);
            case 8: return launch_smallk<8>(M, n, k, A, lda, B, ldb, C, ldc, s, copy_flag, bias);
            case 9: return launch_smallk<9>(M, n, k, A, lda, B, ldb, C, ldc, s, copy_flag, bias);
            default: return launch_smallk<10>(M, n, k, A, lda, B, ldb, C, ldc, s, copy_flag, bias);
        }
    }
    if (N <= 16) return launch_cfg<128, 16, 4, 2>(trans_a, M, N, K, A, lda, B, ldb, C, ldc, splits, split_stride, s, copy_flag, bias);
    if (N <= 32) return launch_cfg<128, 32, 4, 4>(trans_a, M, N, K, A, lda, B, ldb, C, ldc, splits, split_stride, s, copy_flag, bias);
    if (N <= 64) return launch_cfg<128, 64, 8, 4>(trans_a, M, N, K, A, lda, B, ldb, C, ldc, splits, split_stride, s, copy_flag, bias);
    return launch_cfg<128, 128, 8, 8>(trans_a, M, N, K, A, lda, B, ldb, C, ldc, splits, split_stride, s, copy_flag, bias);
}

}  // namespace rpca

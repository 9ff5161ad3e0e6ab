// Passes over A on the tcgen05 tensor cores in split BF16 ("precision form").
//
// The products A X (Section 2's sketch and the A half of every power
// iteration) and A^T Q (the A^* half and B^* = A_c^* Q of Eq. i2) stream the
// FP32 matrix A once per pass.  Each element is split as a = a_hi + a_lo with
// a_hi = bf16(a), a_lo = bf16(a - a_hi) (16 significant bits in all); the
// block operand (X or Q) is split the same way, and three BF16 products
// a_hi b_hi + a_hi b_lo + a_lo b_hi accumulate in FP32 in tensor memory.
//
// Persistent kernel, one CTA per SM, looping over 128-row output tiles (rows
// of A for A X; (column tile, K split) pairs for A^T Q), all N <= 256 output
// columns per tile:
//   warp 0       TMA loads of FP32 A stages (128B-swizzled 32-column boxes),
//                3-stage ring
//   warp 2       bulk copies of the pre-split BF16 block-operand stages
//   warps 8..15  split each FP32 stage into BF16 hi/lo in the MMA's canonical
//                K-major layout (transposing for A^T); the swizzle keeps these
//                shared-memory reads free of bank conflicts
//   warp 1       TMEM allocation (two accumulators); one lane issues the MMAs
//   warps 4..7   epilogue: tcgen05.ld of one accumulator while the MMAs fill
//                the other, FP32 stores
// Every wait on an mbarrier is bounded; a wait that runs out records
// RPCA_ERR_TIMEOUT in the status block and the CTA drains and exits.
//
// The same kernel serves the tall-skinny products of the renormalisations
// (Gram matrices Y^T Y and Y R^-1) with a three-piece split a = hi + mid + lo
// (exact) and the six products of order <= 2^-18, which is as accurate as FP32
// arithmetic: for the Gram the converted tile of Y is both MMA operands.
#include "internal.cuh"
#include "tc_gemm.cuh"
#include "tc_ptx.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

namespace rpca {

namespace {

using namespace ptx;

constexpr int kBM = 128;              // MMA M and CTA output rows
// The tensor cores' FP32 accumulation does not round to nearest: the sums drift
// toward zero by about 2^-27 per accumulated K element (measured: -1.5e-4 relative
// after K = 20000, -1.6e-3 after K = 200000).  Each TMEM accumulation chain
// therefore covers at most kChunkRows of K; the epilogue adds the chunks of a tile
// in FP32 with round-to-nearest, which bounds the drift near 1.5e-5.
constexpr int kChunkRows = 2048;
constexpr int kStagesA = 3;           // FP32 A ring depth
constexpr int kBufs = 2;              // converted BF16 buffers
// A in tensor memory (AT): the converted pieces of A leave shared memory, and the
// block operand gets a ring of its own, so that its copies (from L2) run ahead of
// the MMAs instead of waiting for the buffer the converted A shares with them
constexpr int kStagesAT = 3;          // FP32 A ring
constexpr int kBufsAT = 4;            // converted A buffers in tensor memory (with two N <= 128 accumulators: 512 columns)
constexpr int kBBufsAT = 4;           // block-operand ring
template <bool AT>
struct Ring {
    static constexpr int stages = AT ? kStagesAT : kStagesA;
    static constexpr int bufs = AT ? kBufsAT : kBufs;
    static constexpr int bbufs = AT ? kBBufsAT : kBufs;   // without AT: the converted buffers
};

// Shared-memory plan of one CTA (byte offsets from a 1024-aligned base).  NS BF16
// pieces per operand; GRAM: the B operand is the A operand (no B buffers); AT: the
// pieces of A are in tensor memory (buffers hold B only).
template <int BK, int NS, bool GRAM, bool AT = false>
struct Plan {
    static constexpr uint32_t a32_bytes = kBM * BK * 4;          // FP32 stage
    static constexpr uint32_t abf_bytes = kBM * BK * 2;          // one piece of A
    uint32_t b_bytes;                                            // one piece of B (N x BK bf16)
    uint32_t off_a32, off_buf, buf_bytes, off_bar, total;
    __host__ __device__ explicit Plan(int N) {
        b_bytes = GRAM ? 0u : (uint32_t)N * BK * 2;
        off_a32 = 0;
        off_buf = Ring<AT>::stages * a32_bytes;
        buf_bytes = (AT ? 0u : NS * abf_bytes) + NS * b_bytes;
        off_bar = off_buf + Ring<AT>::bbufs * buf_bytes;
        total = off_bar + 256;
    }
};

struct TcArgs {
    const __nv_bfloat16 *bsplit;  // pre-split block operand: per stage [hi | lo], each N x BK
    float *out;                   // output (+ split * split_stride)
    int64_t out_rows;             // rows of the output that exist (m for A X, n for A^T Q)
    int64_t ldo;                  // leading dimension of out
    int ncols_store;              // columns to store (lp)
    int N;                        // MMA N (multiple of 16, <= 256)
    int64_t per_split;            // K rows per split (A^T Q), K for A X
    int64_t K;                    // total K (n for A X, m for A^T Q)
    int64_t split_stride;         // elements between output partials
    int row_tiles;                // 128-row output tiles
    int ntiles;                   // row_tiles x splits
    DevStatus *st;
    int chunk_st;                 // K stages per TMEM accumulation chain
    const int *skip;              // optional: the launch does nothing when *skip == 0
    const float *bias;            // optional (A X only): out = A X - 1 bias (implicit centring)
    // A X only: row tiles >= full_tiles (the last, partial wave of a persistent grid)
    // are split along K into pieces of tail_per rows, written to tail_part (piece s
    // at s * tail_stride, rows from full_tiles * 128) and summed by tail_sum_kernel
    int full_tiles = 0x7fffffff;
    int64_t tail_per = 0;
    int64_t tail_stride = 0;
    float *tail_part = nullptr;
};

constexpr int kThreads = 512;     // 16 warps
constexpr int kConvWarps = 8;     // warps 8..15
constexpr int kEpiWarp0 = 4;      // warps 4..7

// ADJ = false: out[128 rows of A] = A X.  ADJ = true: out[128 columns of A] = A^T Q
// over the rows of one split (GRAM: Q = A, N <= 128).  Persistent: CTA b takes
// tiles b, b + gridDim.x, ...  AT: the converters write the pieces of A to tensor
// memory (tcgen05.st; two warps per lane quarter, one K half each) and the MMAs read
// A from there (N <= 128, so that two accumulators and the A buffers fit 512 columns).
template <int BK, bool ADJ, int NS, bool GRAM, bool AT = false>
__global__ void __launch_bounds__(kThreads, 1) tc_pass_kernel(const __grid_constant__ CUtensorMap tmap, TcArgs args) {
    static_assert(NS == 2 || NS == 3, "two or three BF16 pieces");
    static_assert(!GRAM || ADJ, "the Gram form is an adjoint product");
    static_assert(!AT || (NS == 2 && !GRAM && BK == 64 && kConvWarps == 8), "tensor-memory A: the split passes");
    constexpr int kSA = Ring<AT>::stages, kNB = Ring<AT>::bufs, kNBB = Ring<AT>::bbufs;
    if (args.skip && *args.skip == 0) return;                  // uniform: before any setup
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const Plan<BK, NS, GRAM, AT> P(args.N);
    uint64_t *full_a = reinterpret_cast<uint64_t *>(smem + P.off_bar);
    uint64_t *empty_a = full_a + kSA;
    uint64_t *full_c = empty_a + kSA;
    uint64_t *empty_c = full_c + kNB;
    uint64_t *full_b = empty_c + kNB;             // AT: the block-operand ring
    uint64_t *empty_b = full_b + kNBB;
    uint64_t *tm_full = empty_b + kNBB;
    uint64_t *tm_empty = tm_full + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(tm_empty + 2);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int N = args.N;
    const uint32_t acc_cols = N <= 32 ? 32 : N <= 64 ? 64 : N <= 128 ? 128 : 256;
    // two accumulators (AT: then the kNB x NS pieces of A, 32 columns each)
    const uint32_t tmem_cols = AT ? 512u : 2 * acc_cols;
    const uint32_t a_col0 = 2 * acc_cols;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kSA; ++s) { mbar_init(&full_a[s], 1); mbar_init(&empty_a[s], kConvWarps); }
        for (int b = 0; b < kNB; ++b) { mbar_init(&full_c[b], kConvWarps + (GRAM || AT ? 0 : 1)); mbar_init(&empty_c[b], 1); }
        for (int b = 0; b < kNBB; ++b) { mbar_init(&full_b[b], 1); mbar_init(&empty_b[b], 1); }
        for (int a = 0; a < 2; ++a) { mbar_init(&tm_full[a], 1); mbar_init(&tm_empty[a], 4); }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    bool ok = true;

    auto fail = [&]() {
        if (!*abort_flag) {
            *abort_flag = 1;
            atomicAdd(&args.st->timeouts, 1);
            dev_fail(args.st, RPCA_ERR_TIMEOUT);
        }
        ok = false;
    };
    // tile -> (first output row, K range, split)
    auto tile_info = [&](int t, int64_t &row0, int64_t &kbeg, int &nst, int &sp) {
        int rt;
        int64_t span;
        if (!ADJ && t >= args.full_tiles) {
            const int tails = args.row_tiles - args.full_tiles, u = t - args.full_tiles;
            rt = args.full_tiles + u % tails;
            sp = u / tails;
            kbeg = (int64_t)sp * args.tail_per;
            span = args.tail_per;
        } else {
            rt = t % args.row_tiles;
            sp = t / args.row_tiles;
            kbeg = ADJ ? (int64_t)sp * args.per_split : 0;
            span = ADJ ? args.per_split : args.K;
        }
        row0 = (int64_t)rt * kBM;
        const int64_t kend = min(args.K, kbeg + span);
        nst = kend > kbeg ? (int)((kend - kbeg + BK - 1) / BK) : 0;
    };

    if (warp == 0) {
        // ---------------- FP32 A producer (TMA) ----------------
        if (lane == 0) {
            uint32_t g = 0;
            for (int t = blockIdx.x; t < args.ntiles && ok; t += gridDim.x) {
                int64_t row0, kbeg;
                int nst, tsp;
                tile_info(t, row0, kbeg, nst, tsp);
                for (int k = 0; k < nst && ok; ++k, ++g) {
                    const int s = g % kSA;
                    if (g >= kSA && !mbar_wait(&empty_a[s], ((g / kSA) & 1) ^ 1, abort_flag)) { fail(); break; }
                    uint8_t *dst = smem + P.off_a32 + s * P.a32_bytes;
                    mbar_arrive_tx(&full_a[s], P.a32_bytes);
                    const int64_t kk = kbeg + (int64_t)k * BK;
                    if (!ADJ) {
                        for (int b = 0; b < BK / 32; ++b)
                            tma_load_2d(dst + b * (kBM * 128), &tmap, (int)(kk + 32 * b), (int)row0, &full_a[s]);
                    } else {
                        for (int b = 0; b < kBM / 32; ++b)
                            tma_load_2d(dst + b * (BK * 128), &tmap, (int)(row0 + 32 * b), (int)kk, &full_a[s]);
                    }
                }
            }
        }
    } else if (warp == 2) {
        // ---------------- block operand producer (bulk copies) ----------------
        if (!GRAM && lane == 0) {
            uint32_t g = 0;
            for (int t = blockIdx.x; t < args.ntiles && ok; t += gridDim.x) {
                int64_t row0, kbeg;
                int nst, tsp;
                tile_info(t, row0, kbeg, nst, tsp);
                const int64_t stage0 = kbeg / BK;
                for (int k = 0; k < nst && ok; ++k, ++g) {
                    const int b = g % kNBB;
                    uint64_t *fb = AT ? &full_b[b] : &full_c[b];
                    uint64_t *eb = AT ? &empty_b[b] : &empty_c[b];
                    if (g >= kNBB && !mbar_wait(eb, ((g / kNBB) & 1) ^ 1, abort_flag)) { fail(); break; }
                    uint8_t *buf = smem + P.off_buf + b * P.buf_bytes;
                    const __nv_bfloat16 *src = args.bsplit + (size_t)(stage0 + k) * NS * N * BK;
                    mbar_arrive_tx(fb, NS * P.b_bytes);
                    bulk_load(buf + (AT ? 0u : NS * P.abf_bytes), src, NS * P.b_bytes, fb);
                }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t idesc = instr_desc_bf16(kBM, N);
            constexpr uint32_t LBO = 128, SBO = (BK / 8) * 128;
            uint32_t g = 0, i = 0;
            for (int t = blockIdx.x; t < args.ntiles && ok; t += gridDim.x) {
                int64_t row0, kbeg;
                int nst, tsp;
                tile_info(t, row0, kbeg, nst, tsp);
                const int nch = nst > 0 ? (nst + args.chunk_st - 1) / args.chunk_st : 1;
                int k = 0;
                for (int ch = 0; ch < nch && ok; ++ch, ++i) {
                const uint32_t acc = i & 1;
                if (i >= 2 && !mbar_wait(&tm_empty[acc], ((i >> 1) & 1) ^ 1, abort_flag)) { fail(); break; }
                tc_fence_after();
                const uint32_t d = tmem_base + acc * acc_cols;
                const int kend = min(nst, k + args.chunk_st);
                for (int kc = 0; k < kend && ok; ++k, ++kc, ++g) {
                    const int b = g % kNB, bb = AT ? (int)(g % kNBB) : b;
                    if (!mbar_wait(&full_c[b], (g / kNB) & 1, abort_flag)) { fail(); break; }
                    if (AT && !mbar_wait(&full_b[bb], (g / kNBB) & 1, abort_flag)) { fail(); break; }
                    tc_fence_after();
                    const uint32_t base = smem_u32(smem + P.off_buf + bb * P.buf_bytes);
                    // piece p of A at base + p * abf_bytes (AT: tensor-memory columns
                    // a_col0 + (b NS + p) 32); of B after the NS pieces of A (GRAM: B = A)
                    const uint32_t bbase = GRAM ? base : base + (AT ? 0u : NS * P.abf_bytes);
                    const uint32_t bstep = GRAM ? P.abf_bytes : P.b_bytes;
                    const uint32_t ta = tmem_base + a_col0 + (uint32_t)(b * NS) * 32u;
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk) {
                        const uint32_t o = kk * 256;
                        const uint32_t acc0 = (kc > 0 || kk > 0) ? 1u : 0u;
                        // products of order <= 2^-9 (NS = 2) or <= 2^-18 (NS = 3): pieces (i, j), i + j < NS
#pragma unroll
                        for (int q = 0; q < (NS == 2 ? 3 : 6); ++q) {
                            const int pi = NS == 2 ? (q == 2 ? 1 : 0) : (q < 3 ? (q == 2 ? 1 : 0) : q - 3);
                            const int pj = NS == 2 ? (q == 1 ? 1 : 0) : (q < 3 ? (q == 1 ? 1 : 0) : 5 - q);
                            if (AT)
                                umma_bf16_ts(d, ta + (uint32_t)pi * 32u + (uint32_t)kk * 8u,
                                             smem_desc(bbase + pj * bstep + o, LBO, SBO), idesc, q == 0 ? acc0 : 1u);
                            else
                                umma_bf16(d, smem_desc(base + pi * P.abf_bytes + o, LBO, SBO),
                                          smem_desc(bbase + pj * bstep + o, LBO, SBO), idesc, q == 0 ? acc0 : 1u);
                        }
                    }
                    umma_commit(&empty_c[b]);
                    if (AT) umma_commit(&empty_b[bb]);
                }
                if (ok) umma_commit(&tm_full[acc]);
                }
            }
        }
    } else if (warp >= kEpiWarp0 && warp < kEpiWarp0 + 4) {
        // ---------------- epilogue: TMEM lanes 32*(warp%4)..+31 ----------------
        const int q = warp & 3;
        uint32_t i = 0;
        for (int t = blockIdx.x; t < args.ntiles && ok; t += gridDim.x) {
            int64_t row0, kbeg;
            int nst, tsp;
            tile_info(t, row0, kbeg, nst, tsp);
            const int nch = nst > 0 ? (nst + args.chunk_st - 1) / args.chunk_st : 1;
            for (int ch = 0; ch < nch && ok; ++ch, ++i) {
            const uint32_t acc = i & 1;
            if (!mbar_wait(&tm_full[acc], (i >> 1) & 1, abort_flag)) { fail(); break; }
            tc_fence_after();
            const bool tail = !ADJ && t >= args.full_tiles;
            const int sp = tsp;
            const int64_t row = row0 + q * 32 + lane;
            float *const obase = tail ? args.tail_part : args.out;
            const int64_t ostride = tail ? args.tail_stride : args.split_stride;
            float *orow = obase + (int64_t)sp * ostride + (tail ? row - (int64_t)args.full_tiles * kBM : row) * args.ldo;
            const bool live = row < args.out_rows;
            const bool vec = ((reinterpret_cast<uintptr_t>(obase) & 15u) == 0) && (args.ldo % 4 == 0) &&
                             (ostride % 4 == 0);
            for (int c0 = 0; c0 < N; c0 += 16) {
                float v[16];
                if (nst > 0) {
                    tmem_ld16(tmem_base + acc * acc_cols + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
                } else {
#pragma unroll
                    for (int e = 0; e < 16; ++e) v[e] = 0.f;
                }
                if (!ADJ && args.bias && ch == 0 && sp == 0) {
                    // Section 5's implicit centring A*X - ones(m,1)*(c*X), bias = c X
#pragma unroll
                    for (int e = 0; e < 16; ++e)
                        if (c0 + e < args.ncols_store) v[e] -= args.bias[c0 + e];
                }
                if (live) {
                    // chunk 0 stores; later chunks of the tile add in FP32 (round to nearest)
                    if (vec && c0 + 16 <= args.ncols_store) {
#pragma unroll
                        for (int e = 0; e < 16; e += 4) {
                            float4 *p4 = reinterpret_cast<float4 *>(orow + c0 + e);
                            float4 o = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
                            if (ch > 0) {
                                const float4 w = *p4;
                                o.x += w.x; o.y += w.y; o.z += w.z; o.w += w.w;
                            }
                            *p4 = o;
                        }
                    } else {
#pragma unroll
                        for (int e = 0; e < 16; ++e)
                            if (c0 + e < args.ncols_store) orow[c0 + e] = ch > 0 ? orow[c0 + e] + v[e] : v[e];
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tm_empty[acc]);
            }
        }
    } else if (warp >= 16 - kConvWarps) {
        // ---------------- converters ----------------
        const int t0 = threadIdx.x - (16 - kConvWarps) * 32;      // 0..255
        constexpr int nthr = kConvWarps * 32;
        uint32_t g = 0;
        for (int t = blockIdx.x; t < args.ntiles && ok; t += gridDim.x) {
            int64_t row0, kbeg;
            int nst, tsp;
            tile_info(t, row0, kbeg, nst, tsp);
            for (int k = 0; k < nst && ok; ++k, ++g) {
                const int s = g % kSA, b = g % kNB;
                if (!mbar_wait(&full_a[s], (g / kSA) & 1, abort_flag)) { fail(); break; }
                if (g >= kNB && !mbar_wait(&empty_c[b], ((g / kNB) & 1) ^ 1, abort_flag)) { fail(); break; }
                const uint8_t *src = smem + P.off_a32 + s * P.a32_bytes;
                uint8_t *buf = smem + P.off_buf + b * P.buf_bytes;
                if constexpr (AT) {
                    // one row of the MMA's A (a row of A for A X, a column of A for A^T Q)
                    // per thread, the 32 K values of this warp's half of the stage
                    tc_fence_after();
                    const int qd = warp & 3, h = (warp - (16 - kConvWarps)) >> 2;
                    float x[32];
                    if (!ADJ) {
                        const int r = qd * 32 + lane;
                        const uint8_t *row = src + h * (kBM * 128) + r * 128;
#pragma unroll
                        for (int c = 0; c < 8; ++c) {
                            const float4 v = *reinterpret_cast<const float4 *>(row + ((c ^ (r & 7)) << 4));
                            x[4 * c] = v.x; x[4 * c + 1] = v.y; x[4 * c + 2] = v.z; x[4 * c + 3] = v.w;
                        }
                    } else {
                        const uint8_t *box = src + qd * (BK * 128);
#pragma unroll
                        for (int e = 0; e < 32; ++e) {
                            const int ii = h * 32 + e;
                            x[e] = *reinterpret_cast<const float *>(box + ii * 128 + (((lane >> 2) ^ (ii & 7)) << 4) +
                                                                     (lane & 3) * 4);
                        }
                    }
                    uint32_t hi[16], lo[16];
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const __nv_bfloat162 hb = __float22bfloat162_rn(make_float2(x[2 * e], x[2 * e + 1]));
                        const float2 hf = __bfloat1622float2(hb);
                        const __nv_bfloat162 lb =
                            __float22bfloat162_rn(make_float2(x[2 * e] - hf.x, x[2 * e + 1] - hf.y));
                        hi[e] = bf2_bits(hb);
                        lo[e] = bf2_bits(lb);
                    }
                    const uint32_t ta = tmem_base + ((uint32_t)(qd * 32) << 16) + a_col0 + (uint32_t)(b * NS) * 32u +
                                        (uint32_t)h * 16u;
                    tmem_st16(ta, hi);
                    tmem_st16(ta + 32u, lo);
                    tmem_st_wait();
                    tc_fence_before();
                } else {
                // core matrices 16 (M) x BK/8 (K); 8 threads per core matrix (one row each)
                constexpr int tasks = (kBM / 8) * (BK / 8) * 8;
#pragma unroll
                for (int id = t0; id < tasks; id += nthr) {
                    const int rr = id & 7, core = id >> 3;
                    int mi, ki;
                    float x[8];
                    if (!ADJ) {
                        ki = core % (BK / 8);
                        mi = core / (BK / 8);
                        // element (r, kc) of a 128 x 32 box: r*128 + ((kc/4) ^ (r%8))*16 + (kc%4)*4
                        const int r = mi * 8 + rr;
                        const int bx = ki >> 2, c0 = (ki & 3) * 2;
                        const uint8_t *row = src + bx * (kBM * 128) + r * 128;
                        const float4 v0 = *reinterpret_cast<const float4 *>(row + ((c0 ^ (r & 7)) << 4));
                        const float4 v1 = *reinterpret_cast<const float4 *>(row + (((c0 + 1) ^ (r & 7)) << 4));
                        x[0] = v0.x; x[1] = v0.y; x[2] = v0.z; x[3] = v0.w;
                        x[4] = v1.x; x[5] = v1.y; x[6] = v1.z; x[7] = v1.w;
                    } else {
                        // mi fastest, so that the four core matrices of a warp sit in distinct bank groups
                        mi = core % (kBM / 8);
                        ki = core / (kBM / 8);
                        const int j = mi * 8 + rr;
                        const int bx = j >> 5, jc = j & 31;
                        const uint8_t *box = src + bx * (BK * 128);
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const int ii = ki * 8 + e;
                            x[e] = *reinterpret_cast<const float *>(box + ii * 128 + (((jc >> 2) ^ (ii & 7)) << 4) +
                                                                     (jc & 3) * 4);
                        }
                    }
                    const uint32_t off = (uint32_t)(mi * (BK / 8) + ki) * 128 + rr * 16;
                    if (NS == 2) {
                        uint4 hi, lo;
                        split8(x, hi, lo);
                        *reinterpret_cast<uint4 *>(buf + off) = hi;
                        *reinterpret_cast<uint4 *>(buf + P.abf_bytes + off) = lo;
                    } else {
                        uint4 hi, mid, lo;
                        split8x3(x, hi, mid, lo);
                        *reinterpret_cast<uint4 *>(buf + off) = hi;
                        *reinterpret_cast<uint4 *>(buf + P.abf_bytes + off) = mid;
                        *reinterpret_cast<uint4 *>(buf + 2 * P.abf_bytes + off) = lo;
                    }
                }
                }
                fence_async_smem();
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(&empty_a[s]);
                    mbar_arrive(&full_c[b]);
                }
            }
        }
    }

    // Drain: after an abort, give copies that were issued time to land.
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (*abort_flag && threadIdx.x == 0) {
        const long long t0 = clock64();
        while (clock64() - t0 < kWaitCycles / 100) {}
    }
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(tmem_cols)
                     : "memory");
    }
}

// ---------------------------------------------------------------------------
// block operand: FP32 P (rows x ld) -> per stage of BK rows, the NS pieces (hi, lo
// or hi, mid, lo) one after the other, each N x BK BF16 in K-major core matrices
// ((n/8) * (BK/8) + k/8) * 64 + (n%8) * 8 + k%8.
// ---------------------------------------------------------------------------
template <int BK, int NS>
__global__ void __launch_bounds__(256)
split_block_kernel(const float *__restrict__ P, int64_t rows, int ncols, int64_t ld, int N,
                   __nv_bfloat16 *__restrict__ out, int64_t nstages) {
    const int64_t chunks = nstages * (int64_t)(N / 8) * (BK / 8) * 8;     // 16-byte chunks per half
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < chunks;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int rr = (int)(c & 7);
        const int64_t core = c >> 3;
        const int ki = (int)(core % (BK / 8));
        const int64_t t2 = core / (BK / 8);
        const int ni = (int)(t2 % (N / 8));
        const int64_t s = t2 / (N / 8);
        const int col = ni * 8 + rr;
        float x[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int64_t i = s * BK + ki * 8 + e;
            x[e] = (i < rows && col < ncols) ? P[i * ld + col] : 0.f;
        }
        __nv_bfloat16 *base = out + s * NS * (int64_t)N * BK;
        const int64_t off = ((int64_t)(ni * (BK / 8) + ki) * 64 + rr * 8);
        if (NS == 2) {
            uint4 hi, lo;
            split8(x, hi, lo);
            *reinterpret_cast<uint4 *>(base + off) = hi;
            *reinterpret_cast<uint4 *>(base + (int64_t)N * BK + off) = lo;
        } else {
            uint4 hi, mid, lo;
            split8x3(x, hi, mid, lo);
            *reinterpret_cast<uint4 *>(base + off) = hi;
            *reinterpret_cast<uint4 *>(base + (int64_t)N * BK + off) = mid;
            *reinterpret_cast<uint4 *>(base + 2 * (int64_t)N * BK + off) = lo;
        }
    }
}

// Y[rows] = sum over the K pieces of the split tail tiles, in piece order (deterministic).
__global__ void __launch_bounds__(256)
tail_sum_kernel(const float *__restrict__ part, int pieces, int64_t stride, int64_t rows, int ncols, int64_t ldo,
                float *__restrict__ Y) {
    const int64_t total = rows * ncols;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / ncols;
        const int c = (int)(e - r * ncols);
        const int64_t o = r * ldo + c;
        float v = part[o];
        for (int p = 1; p < pieces; ++p) v += part[(int64_t)p * stride + o];
        Y[o] = v;
    }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

int make_map(CUtensorMap *map, const float *A, int64_t m, int64_t n, int64_t lda, uint32_t box_x, uint32_t box_y) {
    auto enc = get_encode();
    if (!enc) return RPCA_ERR_CUDA;
    cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)m};
    cuuint64_t strides[1] = {(cuuint64_t)lda * 4};
    cuuint32_t box[2] = {box_x, box_y};
    cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(A), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? RPCA_OK : RPCA_ERR_CUDA;
}

template <int BK, bool ADJ, int NS = 2, bool GRAM = false, bool AT = false>
int launch_pass(const CUtensorMap &map, const TcArgs &a, dim3 grid, cudaStream_t s) {
    const Plan<BK, NS, GRAM, AT> P(a.N);
    const size_t smem = P.total + 1024;
    auto kern = tc_pass_kernel<BK, ADJ, NS, GRAM, AT>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return RPCA_ERR_CUDA;
    kern<<<grid, kThreads, smem, s>>>(map, a);
    RPCA_CHECK_LAUNCH();
    return RPCA_OK;
}

}  // namespace

int tc_n(int lp) { return (int)round_up(lp, 16); }
int tc_bk(int lp) { return tc_n(lp) <= 128 ? 64 : 32; }

bool tc_supported(const float *A, int64_t lda, int lp) {
    return tc_n(lp) <= 256 && (reinterpret_cast<uintptr_t>(A) & 15u) == 0 && lda % 4 == 0;
}

size_t tc_split_bytes(int64_t rows, int lp) {
    const int N = tc_n(lp), BK = tc_bk(lp);
    return (size_t)cdiv(rows, BK) * 2 * N * BK * sizeof(__nv_bfloat16);
}

int tc_adjoint_splits(int64_t n, int64_t m, int lp) {
    // (column tile, split) work items: with fewer tiles than SMs, about one item per
    // SM; with more, the fewest splits (<= 16) whose items fill >= 90% of the waves
    // of one CTA per SM (157 tiles on 152 SMs would otherwise take two waves)
    const int64_t tiles = cdiv(n, kBM);
    const int64_t stages = cdiv(m, tc_bk(lp));
    const int64_t sms = num_sms();
    int64_t s = 1;
    if (tiles <= sms) {
        s = std::max<int64_t>(1, sms / tiles);
    } else {
        for (s = 1; s < 16; ++s) {
            const int64_t items = tiles * s;
            if ((double)items / (double)(cdiv(items, sms) * sms) >= 0.9) break;
        }
    }
    return (int)std::min<int64_t>(s, std::max<int64_t>(1, stages / 4));
}

int launch_tc_split(const float *P, int64_t rows, int lp, __nv_bfloat16 *out, cudaStream_t s) {
    const int N = tc_n(lp), BK = tc_bk(lp);
    const int64_t nst = cdiv(rows, BK);
    const int64_t chunks = nst * (N / 8) * (BK / 8) * 8;
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(cdiv(chunks, 256), (int64_t)num_sms() * 8));
    if (BK == 64)
        split_block_kernel<64, 2><<<(unsigned)grid, 256, 0, s>>>(P, rows, lp, lp, N, out, nst);
    else
        split_block_kernel<32, 2><<<(unsigned)grid, 256, 0, s>>>(P, rows, lp, lp, N, out, nst);
    RPCA_CHECK_LAUNCH();
    return RPCA_OK;
}

size_t tc_apply_tail_bytes(int lp) { return (size_t)std::max(num_sms(), 1) * kBM * lp * sizeof(float); }

int launch_tc_apply(const float *A, int64_t m, int64_t n, int64_t lda, const __nv_bfloat16 *xsplit, int lp,
                    float *Y, DevStatus *st, cudaStream_t s, const float *bias, float *tail_part) {
    const int N = tc_n(lp), BK = tc_bk(lp);
    CUtensorMap map;
    RPCA_TRY(make_map(&map, A, m, n, lda, 32, kBM));
    const int tiles = (int)cdiv(m, kBM);
    TcArgs a{xsplit, Y, m, lp, lp, N, n, n, 0, tiles, tiles, st, std::max(1, kChunkRows / BK), nullptr, bias};
    // The persistent grid takes the tiles in waves of one per SM.  When the last wave
    // is partial (R tiles), its tiles are split along K into S <= SMs / R pieces of at
    // least four stages, so that the wave takes about 1/S of a tile's time.
    const int sms = num_sms();
    const int R = tiles % sms;
    int pieces = 1;
    if (tail_part && R > 0) {
        const int64_t stages = cdiv(n, BK);
        const int64_t want = std::min<int64_t>(sms / R, stages / 4);
        if (want >= 2) {
            a.tail_per = round_up(cdiv(n, want), BK);
            pieces = (int)cdiv(n, a.tail_per);
        }
    }
    if (pieces >= 2) {
        a.full_tiles = tiles - R;
        a.tail_stride = (int64_t)R * kBM * lp;
        a.tail_part = tail_part;
        a.ntiles = a.full_tiles + R * pieces;
    }
    dim3 grid((unsigned)std::min(a.ntiles, sms), 1, 1);
    // N <= 128 (BK = 64): A in tensor memory
    RPCA_TRY(BK == 64 ? (launch_pass<64, false, 2, false, true>(map, a, grid, s)) : (launch_pass<32, false>(map, a, grid, s)));
    if (pieces >= 2) {
        const int64_t r0 = (int64_t)a.full_tiles * kBM, rows = m - r0;
        const int64_t g = std::max<int64_t>(1, std::min<int64_t>(cdiv(rows * lp, 256), (int64_t)sms * 4));
        tail_sum_kernel<<<(unsigned)g, 256, 0, s>>>(tail_part, pieces, a.tail_stride, rows, lp, lp, Y + r0 * lp);
        RPCA_CHECK_LAUNCH();
    }
    return RPCA_OK;
}

int launch_tc_adjoint(const float *A, int64_t m, int64_t n, int64_t lda, const __nv_bfloat16 *qsplit, int lp,
                      float *part, int splits, DevStatus *st, cudaStream_t s) {
    const int N = tc_n(lp), BK = tc_bk(lp);
    CUtensorMap map;
    RPCA_TRY(make_map(&map, A, m, n, lda, 32, (uint32_t)BK));
    const int64_t per = round_up(cdiv(m, splits), BK);
    const int rt = (int)cdiv(n, kBM);
    TcArgs a{qsplit, part, n, lp, lp, N, per, m, n * (int64_t)lp, rt, rt * splits, st, std::max(1, kChunkRows / BK),
             nullptr};
    dim3 grid((unsigned)std::min(rt * splits, num_sms()), 1, 1);
    return BK == 64 ? launch_pass<64, true, 2, false, true>(map, a, grid, s) : launch_pass<32, true>(map, a, grid, s);
}

// ---------------------------------------------------------------------------
// renormalisation products in three-piece split BF16
// ---------------------------------------------------------------------------
namespace {
constexpr int kRmulBK = 32;             // K stage of Y R^-1 (K = lp is short)

// out = Y when *flag == 0 (a skipped product is the identity), else nothing
__global__ void __launch_bounds__(256) copy_if_skipped_kernel(const int *__restrict__ flag, const float4 *__restrict__ src,
                                                              float4 *__restrict__ dst, int64_t n4) {
    if (*flag != 0) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}
constexpr int kGramChainStages = 4;     // 256 rows per TMEM chain: drift <= 2e-6 on Y^T Y
}  // namespace

bool tc_gram_ok(int64_t rows, int lp) { return rows >= kTcRenormMinRows && tc_n(lp) <= kBM; }
bool tc_rmul_ok(int64_t rows, int ncols) { return rows >= kTcRenormMinRows && tc_n(ncols) <= 256; }

size_t tc_rmul_split_bytes(int lp) {
    return (size_t)cdiv(lp, kRmulBK) * 3 * tc_n(lp) * kRmulBK * sizeof(__nv_bfloat16);
}

int launch_tc_gram(const float *Y, int64_t rows, int lp, float *part, int *splits_out, const int *skip,
                   DevStatus *st, cudaStream_t s) {
    if (!tc_gram_ok(rows, lp)) return RPCA_ERR_INVALID_ARG;
    const int N = tc_n(lp);
    constexpr int BK = 64;
    const int splits = tc_adjoint_splits(lp, rows, lp);
    CUtensorMap map;
    RPCA_TRY(make_map(&map, Y, rows, lp, lp, 32, (uint32_t)BK));
    const int64_t per = round_up(cdiv(rows, splits), BK);
    TcArgs a{nullptr, part, lp, lp, lp, N, per, rows, (int64_t)lp * lp, 1, splits, st, kGramChainStages, skip};
    *splits_out = splits;
    return launch_pass<BK, true, 3, true>(map, a, dim3((unsigned)std::min(splits, num_sms()), 1, 1), s);
}

int launch_tc_rmul(const float *Y, int64_t rows, int lp, const float *R, int64_t ldr, int ncols,
                   __nv_bfloat16 *rsplit, float *out, int64_t ldo, const int *skip, DevStatus *st, cudaStream_t s) {
    if (!tc_rmul_ok(rows, ncols) || ncols > lp) return RPCA_ERR_INVALID_ARG;
    const int N = tc_n(ncols);
    constexpr int BK = kRmulBK;
    const int64_t nst = cdiv(lp, BK);
    const int64_t chunks = nst * (N / 8) * (BK / 8) * 8;
    split_block_kernel<BK, 3><<<(unsigned)cdiv(chunks, 256), 256, 0, s>>>(R, lp, ncols, ldr, N, rsplit, nst);
    RPCA_CHECK_LAUNCH();
    CUtensorMap map;
    RPCA_TRY(make_map(&map, Y, rows, lp, lp, 32, kBM));
    const int tiles = (int)cdiv(rows, kBM);
    TcArgs a{rsplit, out, rows, ldo, ncols, N, lp, lp, 0, tiles, tiles, st, std::max(1, kChunkRows / BK), skip};
    RPCA_TRY((launch_pass<BK, false, 3, false>(map, a, dim3((unsigned)std::min(tiles, num_sms()), 1, 1), s)));
    if (skip) {
        // a skipped round is the identity: out = Y (square R, out shaped like Y)
        if (ncols != lp || ldo != lp) return RPCA_ERR_INVALID_ARG;
        const int64_t n4 = rows * (int64_t)lp / 4;
        const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(cdiv(n4, 256), (int64_t)num_sms() * 4));
        copy_if_skipped_kernel<<<(unsigned)grid, 256, 0, s>>>(skip, reinterpret_cast<const float4 *>(Y),
                                                              reinterpret_cast<float4 *>(out), n4);
        RPCA_CHECK_LAUNCH();
    }
    return RPCA_OK;
}

}  // namespace rpca

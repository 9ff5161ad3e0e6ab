// Batched randomized PCA: many small, uneven dense matrices in one launch
// (device code, included by the translation units that instantiate the kernel).
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
#pragma once

#include "internal.cuh"
#include "philox.cuh"

namespace rpca {

// one matrix of the batch (the layout of rpca_mat_desc)
struct Item {
    const float *A;
    int64_t m, n, lda;
    float *U;
    int64_t ldu;
    float *S;
    float *V;
    int64_t ldv;
};

// arguments of one launch of the batched kernel
struct BatchLaunch {
    const Item *items;
    const int32_t *order;
    int count, l, k, its, raw;
    uint64_t seed;
    const float *const *weights;
    int32_t *item_status;
    const int32_t *active;        // optional: items with active[i] == 0 are skipped (outputs untouched)
    float *sk1;                   // optional: s_{k+1} of each item's rank-l approximation
    int *queue;
    float *slots;
    int64_t slot_floats, max_m;
    int grid;
    cudaStream_t stream;
};

namespace {

constexpr int kThreads = 512;
constexpr int kMaxLP = 40;                 // l <= 32
constexpr int kMaxNL = 24576;              // n * lp floats of the n-side block
// pass tiles: RPT rows (A X) or columns (A^T Y) of A per thread, KB deep; the shapes in use
// are (2, 64), (4, 32) and (8, 32)
constexpr int kJacSweeps = 30;
constexpr int kGramGroups = 16;            // row groups of the Gram
constexpr int kMaxPairs = 64;              // 4x4 blocks of the upper triangle, lp <= 40 -> 55
constexpr int pass_floats(int rpt, int kb) { return kb * (64 * rpt + 4) + kb * kMaxLP; }
constexpr int kPassFloats = pass_floats(8, 32) > pass_floats(2, 64) ? pass_floats(8, 32) : pass_floats(2, 64);
constexpr int kTileFloats = kGramGroups * kMaxPairs * 16 > kPassFloats ? kGramGroups * kMaxPairs * 16 : kPassFloats;

struct Smem {
    float X[kMaxNL];                        // n x lp
    float tile[kTileFloats];
    float G[kMaxLP * kMaxLP];
    float R[kMaxLP * kMaxLP];
    float Racc[kMaxLP * kMaxLP];
    float T[kMaxLP * kMaxLP];
    float vec[4 * kMaxLP];                  // means, sums
    float sig[kMaxLP];
    int perm[kMaxLP];
    int flag;
    int item;
};
// At most 196 KB of shared memory per CTA: past that the SM switches to its largest
// carve-out and the L1 cache left next to it (which serves the m-side block Y) drops
// from ~60 KB to ~28 KB, measured ~10% slower on the kernel-matrix batch.
static_assert(sizeof(Smem) <= 196 * 1024, "batched shared memory beyond the 196 KB carve-out");

// ---------------------------------------------------------------------------
// Test matrix of one item: the single-matrix path's stream keyed (seed, 0), element
// e = i*l + j, scaled by the optional column weights.
// ---------------------------------------------------------------------------
__device__ void gen_omega(Smem &sm, int64_t n, int l, int lp, uint64_t seed, const float *weights) {
    for (int64_t e = threadIdx.x; e < n * lp; e += blockDim.x) sm.X[e] = 0.f;
    __syncthreads();
    const int64_t total = n * (int64_t)l, nblk = (total + 3) / 4;
    for (int64_t b = threadIdx.x; b < nblk; b += blockDim.x) {
        float z[4];
        gauss4((uint64_t)b, seed, 0, z);
        for (int t = 0; t < 4; ++t) {
            const int64_t e = 4 * b + t;
            if (e < total) {
                const int64_t i = e / l;
                const int j = (int)(e - i * l);
                sm.X[i * lp + j] = weights ? z[t] * weights[i] : z[t];
            }
        }
    }
    __syncthreads();
}

// RPT consecutive floats of a shared-memory row (16- or 8-byte aligned), into registers
template <int RPT>
__device__ __forceinline__ void load_run(const float *p, float (&v)[RPT]) {
    if constexpr (RPT % 4 == 0) {
#pragma unroll
        for (int a = 0; a < RPT; a += 4) {
            const float4 t = *reinterpret_cast<const float4 *>(p + a);
            v[a] = t.x; v[a + 1] = t.y; v[a + 2] = t.z; v[a + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int a = 0; a < RPT; a += 2) {
            const float2 t = *reinterpret_cast<const float2 *>(p + a);
            v[a] = t.x; v[a + 1] = t.y;
        }
    }
}

// Y (m x lp, global) = A X (X = sm.X, n x lp).  Thread: RPT rows x CPT columns (tiles of
// 64 RPT rows); the next A tile is fetched into registers while the current one is
// multiplied.  Every output sums over k in order whatever RPT is.
template <int CPT, int RPT, int KB>
__device__ void apply_ax(Smem &sm, const float *__restrict__ A, int64_t m, int64_t n, int64_t lda, int lp,
                         float *__restrict__ Y) {
    constexpr int BM = 64 * RPT, LDT = BM + 4;
    float *As = sm.tile;                          // [KB][LDT]
    const int tid = threadIdx.x;
    const int rq = tid >> 3, cg = tid & 7;        // 64 row groups x 8 column groups
    constexpr int PER = BM * KB / kThreads;      // elements of a tile per thread
    float pre[PER];
    auto fetch = [&](int64_t r0, int64_t k0) {
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int e = tid + q * kThreads;
            const int r = e / KB, kk = e % KB;
            const int64_t gr = r0 + r, gk = k0 + kk;
            pre[q] = (gr < m && gk < n) ? __ldg(A + gr * lda + gk) : 0.f;
        }
    };
    auto stash = [&]() {
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int e = tid + q * kThreads;
            As[(e % KB) * LDT + e / KB] = pre[q];
        }
    };
    const int64_t ktiles = (n + KB - 1) / KB;
    for (int64_t r0 = 0; r0 < m; r0 += BM) {
        float acc[RPT][CPT];
#pragma unroll
        for (int a = 0; a < RPT; ++a)
#pragma unroll
            for (int q = 0; q < CPT; ++q) acc[a][q] = 0.f;
        fetch(r0, 0);
        for (int64_t t = 0; t < ktiles; ++t) {
            const int64_t k0 = t * KB;
            __syncthreads();
            stash();
            __syncthreads();
            if (t + 1 < ktiles) fetch(r0, k0 + KB);
            const int kn = (int)min((int64_t)KB, n - k0);
            for (int kk = 0; kk < kn; ++kk) {
                float a[RPT];
                load_run<RPT>(&As[kk * LDT + RPT * rq], a);
                const float *xr = sm.X + (k0 + kk) * lp;
#pragma unroll
                for (int q = 0; q < CPT; ++q) {
                    const int c = cg + 8 * q;
                    const float x = c < lp ? xr[c] : 0.f;
#pragma unroll
                    for (int u = 0; u < RPT; ++u) acc[u][q] = fmaf(a[u], x, acc[u][q]);
                }
            }
        }
#pragma unroll
        for (int a = 0; a < RPT; ++a) {
            const int64_t r = r0 + RPT * rq + a;
            if (r < m)
#pragma unroll
                for (int q = 0; q < CPT; ++q) {
                    const int c = cg + 8 * q;
                    if (c < lp) Y[r * lp + c] = acc[a][q];
                }
        }
    }
    __syncthreads();
}

// X (n x lp, shared) = A^T Y (Y global, m x lp).  Thread: RPT columns of A x CPT columns of
// Y (tiles of 64 RPT columns); the next tiles are fetched into registers while the current
// ones are multiplied.  Every output sums over the rows in order whatever RPT is.
template <int CPT, int RPT, int KB>
__device__ void apply_aty(Smem &sm, const float *__restrict__ A, int64_t m, int64_t n, int64_t lda, int lp,
                          const float *__restrict__ Y) {
    constexpr int BN = 64 * RPT, LDT = BN + 4;
    float *As = sm.tile;                          // [KB][LDT]
    float *Ys = sm.tile + KB * LDT;              // [KB][lp]
    const int tid = threadIdx.x;
    const int cq = tid >> 3, cg = tid & 7;        // 64 column groups of A x 8 column groups of Y
    constexpr int PER = BN * KB / kThreads;
    float pre[PER], prey[(KB * kMaxLP + kThreads - 1) / kThreads];
    auto fetch = [&](int64_t c0, int64_t r0) {
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int e = tid + q * kThreads;
            const int rr = e / BN, cc = e % BN;
            const int64_t gr = r0 + rr, gc = c0 + cc;
            pre[q] = (gr < m && gc < n) ? __ldg(A + gr * lda + gc) : 0.f;
        }
#pragma unroll
        for (int q = 0; q < (KB * kMaxLP + kThreads - 1) / kThreads; ++q) {
            const int e = tid + q * kThreads;
            float v = 0.f;
            if (e < KB * lp) {
                const int rr = e / lp;
                const int64_t gr = r0 + rr;
                if (gr < m) v = Y[gr * lp + (e - rr * lp)];
            }
            prey[q] = v;
        }
    };
    auto stash = [&]() {
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int e = tid + q * kThreads;
            As[(e / BN) * LDT + e % BN] = pre[q];
        }
#pragma unroll
        for (int q = 0; q < (KB * kMaxLP + kThreads - 1) / kThreads; ++q) {
            const int e = tid + q * kThreads;
            if (e < KB * lp) Ys[e] = prey[q];
        }
    };
    const int64_t rtiles = (m + KB - 1) / KB;
    for (int64_t c0 = 0; c0 < n; c0 += BN) {
        float acc[RPT][CPT];
#pragma unroll
        for (int a = 0; a < RPT; ++a)
#pragma unroll
            for (int q = 0; q < CPT; ++q) acc[a][q] = 0.f;
        fetch(c0, 0);
        for (int64_t t = 0; t < rtiles; ++t) {
            const int64_t r0 = t * KB;
            __syncthreads();
            stash();
            __syncthreads();
            if (t + 1 < rtiles) fetch(c0, r0 + KB);
            const int kn = (int)min((int64_t)KB, m - r0);
            for (int kk = 0; kk < kn; ++kk) {
                float a[RPT];
                load_run<RPT>(&As[kk * LDT + RPT * cq], a);
                const float *yr = Ys + kk * lp;
#pragma unroll
                for (int q = 0; q < CPT; ++q) {
                    const int c = cg + 8 * q;
                    const float y = c < lp ? yr[c] : 0.f;
#pragma unroll
                    for (int u = 0; u < RPT; ++u) acc[u][q] = fmaf(a[u], y, acc[u][q]);
                }
            }
        }
#pragma unroll
        for (int a = 0; a < RPT; ++a) {
            const int64_t col = c0 + RPT * cq + a;
            if (col < n)
#pragma unroll
                for (int q = 0; q < CPT; ++q) {
                    const int c = cg + 8 * q;
                    if (c < lp) sm.X[col * lp + c] = acc[a][q];
                }
        }
    }
    __syncthreads();
}

// Column sums of B (rows x lp, global or shared) for c < l, in fixed order: vec[off + c].
__device__ void col_sums(Smem &sm, const float *B, int64_t rows, int l, int lp, int off) {
    float *part = sm.tile;                        // [16][lp]
    const int g = threadIdx.x / 32, c = threadIdx.x % 32;   // 16 row groups x 32 columns
    for (int cb = 0; cb < l; cb += 32) {
        float s = 0.f;
        if (cb + c < l)
            for (int64_t r = g; r < rows; r += 16) s += B[r * lp + cb + c];
        __syncthreads();
        if (cb + c < lp) part[g * lp + cb + c] = s;
        __syncthreads();
        if (threadIdx.x < 32 && cb + c < l) {
            float t = 0.f;
            for (int q = 0; q < 16; ++q) t += part[q * lp + cb + c];
            sm.vec[off + cb + c] = t;
        }
    }
    __syncthreads();
}

// G (l x l, shared) = B^T B over rows (B global or shared, ld lp, 16-byte aligned rows).
// 16 row groups of 32 threads; a thread owns up to two 4x4 blocks (bi <= bj) of the upper
// triangle and accumulates them over its group's rows; partials summed in group order.
__device__ void gram(Smem &sm, const float *B, int64_t rows, int l, int lp) {
    float *part = sm.tile;                        // [kGramGroups][kMaxPairs][16]
    const int nb = lp / 4, npairs = nb * (nb + 1) / 2;
    const int g = threadIdx.x / 32, lane = threadIdx.x % 32;
    int bi[2], bj[2];
    bool live[2];
    for (int q = 0; q < 2; ++q) {
        int p = lane + 32 * q;
        live[q] = p < npairs;
        if (!live[q]) p = 0;
        int i = 0;
        while (p >= nb - i) { p -= nb - i; ++i; }
        bi[q] = i;
        bj[q] = i + p;
    }
    float acc[2][4][4];
    for (int q = 0; q < 2; ++q)
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) acc[q][a][b] = 0.f;
    for (int64_t r = g; r < rows; r += kGramGroups) {
        const float *row = B + r * lp;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            if (!live[q]) continue;
            const float4 a = *reinterpret_cast<const float4 *>(row + 4 * bi[q]);
            const float4 b = *reinterpret_cast<const float4 *>(row + 4 * bj[q]);
            const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) acc[q][x][y] = fmaf(av[x], bv[y], acc[q][x][y]);
        }
    }
    for (int q = 0; q < 2; ++q)
        if (live[q])
            for (int e = 0; e < 16; ++e) part[(g * kMaxPairs + lane + 32 * q) * 16 + e] = acc[q][e / 4][e % 4];
    __syncthreads();
    for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
        const int a = e / l, b = e % l;
        const int i = min(a, b) / 4, j = max(a, b) / 4;
        const int x = (a <= b ? a : b) % 4, y = (a <= b ? b : a) % 4;
        // pair index of (i, j): rows 0..i-1 contribute nb - r pairs each
        const int p = i * nb - i * (i - 1) / 2 + (j - i);
        // within the block (i, j) the entry is acc[x][y] with x from block i, y from block j;
        // on a diagonal block (i == j) both orders hold the same value
        float t = 0.f;
        for (int q = 0; q < kGramGroups; ++q) t += part[(q * kMaxPairs + p) * 16 + x * 4 + y];
        sm.G[e] = t;
    }
    __syncthreads();
}

// Cholesky G = R^T R (one warp; R upper in sm.R), shifted on collapse.  Returns via sm.flag
// whether a shift was needed.
__device__ void cholesky(Smem &sm, int l) {
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        float maxd = 0.f;
        for (int j = 0; j < l; ++j) maxd = fmaxf(maxd, sm.G[j * l + j]);
        const float tau = 16.f * (float)l * 0x1p-24f;
        float shift = 0.f;
        bool ok = false;
        for (int attempt = 0; attempt < 4 && !ok; ++attempt) {
            for (int e = lane; e < l * l; e += 32) sm.R[e] = sm.G[e] + ((e / l == e % l) ? shift : 0.f);
            __syncwarp();
            ok = true;
            for (int j = 0; j < l; ++j) {
                const float d = sm.R[j * l + j];
                if (!(d > tau * sm.G[j * l + j] + 0.5f * shift) || !(d > 0.f)) { ok = false; break; }
                const float r = sqrtf(d);
                __syncwarp();
                if (lane > j && lane < l) sm.R[j * l + lane] /= r;
                if (lane == j) sm.R[j * l + j] = r;
                __syncwarp();
                if (lane > j && lane < l)
                    for (int i = j + 1; i <= lane; ++i) sm.R[i * l + lane] -= sm.R[j * l + i] * sm.R[j * l + lane];
                __syncwarp();
            }
            if (!ok) shift = (shift == 0.f) ? 16.f * (float)l * 0x1p-24f * fmaxf(maxd, 1e-30f) : shift * 100.f;
        }
        for (int e = lane; e < l * l; e += 32)
            if (e / l > e % l) sm.R[e] = 0.f;
        if (!ok)
            for (int e = lane; e < l * l; e += 32) sm.R[e] = (e / l == e % l) ? 1.f : 0.f;
        if (lane == 0) sm.flag = shift != 0.f ? 1 : 0;
    }
    __syncthreads();
}

// B <- B R^-1 row by row (forward substitution z R = b, in place), columns < l.
__device__ void solve_rows(Smem &sm, float *B, int64_t rows, int l, int lp) {
    for (int64_t r = threadIdx.x; r < rows; r += blockDim.x) {
        float *b = B + r * lp;
        for (int j = 0; j < l; ++j) {
            float s = b[j];
            for (int i = 0; i < j; ++i) s = fmaf(-b[i], sm.R[i * l + j], s);
            b[j] = s / sm.R[j * l + j];
        }
    }
    __syncthreads();
}

// Racc <- R Racc (upper triangular, l x l); first = true sets Racc = R.
__device__ void accumulate_r(Smem &sm, int l, bool first) {
    for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
        const int i = e / l, k = e % l;
        float v = 0.f;
        if (first) v = sm.R[e];
        else if (k >= i)
            for (int t = i; t <= k; ++t) v = fmaf(sm.R[i * l + t], sm.Racc[t * l + k], v);
        sm.T[e] = v;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < l * l; e += blockDim.x) sm.Racc[e] = sm.T[e];
    __syncthreads();
}

// CholeskyQR round on B (rows x lp) in place; returns whether it shifted.
__device__ bool cholqr(Smem &sm, float *B, int64_t rows, int l, int lp) {
    gram(sm, B, rows, l, lp);
    cholesky(sm, l);
    const bool shifted = sm.flag != 0;
    solve_rows(sm, B, rows, l, lp);
    return shifted;
}

// One-sided Jacobi on M = Racc^T (columns j of M = rows of Racc), 16 warps, one pair each
// per round-robin step.  Leaves sigma (descending) in sm.sig, W (l x l, column r =
// r-th left vector) in sm.G and Z (right vectors) in sm.R, both sorted.
__device__ void small_svd(Smem &sm, int l) {
    float *M = sm.T;                                // M[j][i] = column j, row i (= Racc[j][i])
    float *Z = sm.R;                                // Z[j][i] = column j of Z
    for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
        M[e] = sm.Racc[e];
        Z[e] = (e / l == e % l) ? 1.f : 0.f;
    }
    __syncthreads();
    const int L = l + (l & 1), npairs = L / 2;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const float tol = 8.f * sqrtf((float)l) * 0x1p-24f;
    for (int sweep = 0; sweep < kJacSweeps; ++sweep) {
        if (threadIdx.x == 0) sm.flag = 0;
        __syncthreads();
        for (int step = 0; step < L - 1; ++step) {
            for (int g = warp; g < npairs; g += blockDim.x / 32) {
                auto player = [&](int pos) { return pos == 0 ? 0 : 1 + (pos - 1 + step) % (L - 1); };
                const int a0 = player(g), b0 = player(L - 1 - g);
                const int p = min(a0, b0), q = max(a0, b0);
                float x = 0.f, y = 0.f;
                if (q < l && lane < l) { x = M[p * l + lane]; y = M[q * l + lane]; }
                float al = x * x, be = y * y, ga = x * y;
                for (int off = 16; off > 0; off >>= 1) {
                    al += __shfl_xor_sync(0xffffffffu, al, off);
                    be += __shfl_xor_sync(0xffffffffu, be, off);
                    ga += __shfl_xor_sync(0xffffffffu, ga, off);
                }
                if (q < l && fabsf(ga) > tol * sqrtf(al * be) && ga != 0.f) {
                    const float zeta = (be - al) / (2.f * ga);
                    const float t = copysignf(1.f, zeta) / (fabsf(zeta) + hypotf(zeta, 1.f));
                    const float cs = rsqrtf(fmaf(t, t, 1.f)), sn = cs * t;
                    if (lane < l) {
                        M[p * l + lane] = cs * x - sn * y;
                        M[q * l + lane] = sn * x + cs * y;
                        const float zx = Z[p * l + lane], zy = Z[q * l + lane];
                        Z[p * l + lane] = cs * zx - sn * zy;
                        Z[q * l + lane] = sn * zx + cs * zy;
                    }
                    if (lane == 0) sm.flag = 1;
                }
            }
            __syncthreads();
        }
        const int rot = sm.flag;
        __syncthreads();
        if (!rot) break;
    }
    // sigma_j = |M_j| / |Z_j|: the rotations are orthogonal only to a few ulps with a
    // systematic sign and scale M_j and Z_j alike, so the ratio and Z_j / |Z_j| remove
    // that drift; rank descending (ties by index).  sm.sig holds 1 / |Z_j| meanwhile.
    if (threadIdx.x < l) {
        const int j = threadIdx.x;
        float s2 = 0.f, z2 = 0.f;
        for (int i = 0; i < l; ++i) {
            s2 = fmaf(M[j * l + i], M[j * l + i], s2);
            z2 = fmaf(Z[j * l + i], Z[j * l + i], z2);
        }
        const float iz = z2 > 0.f ? 1.f / sqrtf(z2) : 1.f;
        sm.vec[j] = sqrtf(s2) * iz;
        sm.sig[j] = iz;
    }
    __syncthreads();
    if (threadIdx.x < l) {
        const int j = threadIdx.x;
        const float sj = sm.vec[j];
        int rank = 0;
        for (int i = 0; i < l; ++i) rank += (sm.vec[i] > sj) || (sm.vec[i] == sj && i < j);
        sm.perm[rank] = j;
    }
    __syncthreads();
    // W[:, r] = M_{perm[r]} / |M_{perm[r]}| (stored as G[i * l + r]);  Zs[:, r] = Z_{perm[r]} / |Z_{perm[r]}|
    // (stored in Racc)
    for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
        const int i = e / l, r = e % l;
        const int j = sm.perm[r];
        const float s = sm.vec[j], iz = sm.sig[j];
        sm.G[i * l + r] = s > 0.f ? M[j * l + i] * iz / s : 0.f;
        sm.Racc[i * l + r] = Z[j * l + i] * iz;
    }
    __syncthreads();
    if (threadIdx.x < l) sm.sig[threadIdx.x] = sm.vec[sm.perm[threadIdx.x]];
    __syncthreads();
}

// Per item: the method.  Y0 / Y1: this CTA's m-side slots.
template <int CPT, int RPT, int KB>
__device__ void run_item(Smem &sm, const Item &it, int l, int lp, int k, int its, int raw, uint64_t seed,
                         const float *weights, float *Y0, int32_t *status, float *sk1_out) {
    const float *A = it.A;
    const int64_t m = it.m, n = it.n, lda = it.lda;
    float *mean = sm.vec + kMaxLP, *qsum = sm.vec + 2 * kMaxLP;

    // centring of an m-side block: subtract column means (A_c X = A X - 1 (c X)), pad column l = 1
    auto centre_m = [&](float *Y) {
        if (!raw) {
            col_sums(sm, Y, m, l, lp, kMaxLP);
            for (int c = threadIdx.x; c < l; c += blockDim.x) mean[c] /= (float)m;
            __syncthreads();
            for (int64_t e = threadIdx.x; e < m * lp; e += blockDim.x) {
                const int c = (int)(e % lp);
                if (c < l) Y[e] -= mean[c];
            }
            __syncthreads();
        }
    };
    auto pad_m = [&](float *Y) {
        for (int64_t r = threadIdx.x; r < m; r += blockDim.x)
            for (int c = l; c < lp; ++c) Y[r * lp + c] = (c == l && !raw) ? 1.f : 0.f;
        __syncthreads();
        if (!raw) col_sums(sm, Y, m, l, lp, 2 * kMaxLP);
    };
    // X = A_c^T Y: the ones column l of Y gives m c; subtract c (1^T Y)
    auto adjoint = [&](const float *Y) {
        apply_aty<CPT, RPT, KB>(sm, A, m, n, lda, lp, Y);
        if (!raw) {
            for (int64_t e = threadIdx.x; e < n * lp; e += blockDim.x) {
                const int64_t j = e / lp;
                const int c = (int)(e - j * lp);
                if (c < l) sm.X[e] -= (sm.X[j * lp + l] / (float)m) * qsum[c];
            }
            __syncthreads();
        }
        for (int64_t e = threadIdx.x; e < n * lp; e += blockDim.x)
            if ((int)(e % lp) >= l) sm.X[e] = 0.f;
        __syncthreads();
    };

    gen_omega(sm, n, l, lp, seed, weights);
    apply_ax<CPT, RPT, KB>(sm, A, m, n, lda, lp, Y0);
    centre_m(Y0);
    for (int it2 = 0; it2 <= its; ++it2) {
        const bool final_ = it2 == its;
        if (!final_) {
            // implicit renormalisation: X = (A_c^T Y) R^-1
            gram(sm, Y0, m, l, lp);
            cholesky(sm, l);
            pad_m(Y0);
            adjoint(Y0);
            solve_rows(sm, sm.X, n, l, lp);
            cholqr(sm, sm.X, n, l, lp);
            apply_ax<CPT, RPT, KB>(sm, A, m, n, lda, lp, Y0);
            centre_m(Y0);
        } else {
            const bool sh = cholqr(sm, Y0, m, l, lp);
            cholqr(sm, Y0, m, l, lp);
            if (sh) cholqr(sm, Y0, m, l, lp);
            pad_m(Y0);
        }
    }
    // B^* = A_c^* Q; B^* = Q2 R; R^T = W Sigma Z^T
    adjoint(Y0);
    bool sh = cholqr(sm, sm.X, n, l, lp);
    accumulate_r(sm, l, true);
    cholqr(sm, sm.X, n, l, lp);
    accumulate_r(sm, l, false);
    if (sh) {
        cholqr(sm, sm.X, n, l, lp);
        accumulate_r(sm, l, false);
    }
    small_svd(sm, l);          // W in G, Z (sorted) in Racc
    // V = Q2 Z_k with the sign rule on V; U = Q W_k
    float *sgn = sm.vec + 3 * kMaxLP;
    for (int r = threadIdx.x / 32; r < k; r += blockDim.x / 32) {
        const int lane = threadIdx.x % 32;
        float best = -1.f, val = 0.f;
        int64_t bi = 0;
        for (int64_t i = lane; i < n; i += 32) {
            float v = 0.f;
            for (int t = 0; t < l; ++t) v = fmaf(sm.X[i * lp + t], sm.Racc[t * l + r], v);
            if (fabsf(v) > best) { best = fabsf(v); bi = i; val = v; }
        }
        for (int off = 16; off > 0; off >>= 1) {
            const float ob = __shfl_xor_sync(0xffffffffu, best, off);
            const int64_t oi = __shfl_xor_sync(0xffffffffu, bi, off);
            const float ov = __shfl_xor_sync(0xffffffffu, val, off);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; val = ov; }
        }
        if (lane == 0) sgn[r] = val < 0.f ? -1.f : 1.f;
    }
    __syncthreads();
    for (int64_t e = threadIdx.x; e < n * k; e += blockDim.x) {
        const int64_t i = e / k;
        const int r = (int)(e - i * k);
        float v = 0.f;
        for (int t = 0; t < l; ++t) v = fmaf(sm.X[i * lp + t], sm.Racc[t * l + r], v);
        it.V[i * it.ldv + r] = sgn[r] * v;
    }
    for (int64_t e = threadIdx.x; e < m * k; e += blockDim.x) {
        const int64_t i = e / k;
        const int r = (int)(e - i * k);
        float v = 0.f;
        for (int t = 0; t < l; ++t) v = fmaf(Y0[i * lp + t], sm.G[t * l + r], v);
        it.U[i * it.ldu + r] = sgn[r] * v;
    }
    for (int r = threadIdx.x; r < k; r += blockDim.x) it.S[r] = sm.sig[r];
    if (threadIdx.x == 0 && sk1_out) *sk1_out = l > k ? sm.sig[k] : 0.f;     // s_{k+1} of the rank-l approximation
    if (threadIdx.x == 0 && status) *status = RPCA_OK;
    __syncthreads();
}

__device__ __forceinline__ bool item_ok(const Item &it, int l, int k, int64_t max_m) {
    const int lp = (int)round_up(l + 1, 8);
    return it.A && it.U && it.S && it.V && it.m >= 1 && it.n >= 1 && it.m <= max_m && it.lda >= it.n &&
           it.ldu >= k && it.ldv >= k && l <= it.m && l <= it.n && it.n * lp <= kMaxNL &&
           (reinterpret_cast<uintptr_t>(it.A) & 3u) == 0;
}

template <int CPT, int RPT, int KB>
__global__ void __launch_bounds__(kThreads, 1)
batched_kernel(const Item *__restrict__ items, const int32_t *__restrict__ order, int count, int l, int k, int its,
               int raw, uint64_t seed, const float *const *__restrict__ weights, int32_t *__restrict__ item_status,
               const int32_t *__restrict__ active, float *__restrict__ sk1, int *__restrict__ queue,
               float *__restrict__ slots, int64_t slot_floats, int64_t max_m) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
    const int lp = (int)round_up(l + 1, 8);
    float *Y0 = slots + (int64_t)blockIdx.x * slot_floats;
    for (;;) {
        if (threadIdx.x == 0) sm.item = atomicAdd(queue, 1);
        __syncthreads();
        const int q = sm.item;
        __syncthreads();
        if (q >= count) break;
        const int idx = order ? order[q] : q;
        const Item it = items[idx];
        if (!item_ok(it, l, k, max_m)) continue;          // reported by check_items_kernel
        if (active && active[idx] == 0) continue;
        run_item<CPT, RPT, KB>(sm, it, l, lp, k, its, raw, seed, weights ? weights[idx] : nullptr, Y0,
                      item_status ? item_status + idx : nullptr, sk1 ? sk1 + idx : nullptr);
    }
}

}  // namespace

// One launch of the batched kernel with pass tiles of RPT rows (or columns) of A per
// thread, KB deep; the column count per thread follows from l.
template <int RPT, int KB>
int launch_batched_rpt(const BatchLaunch &a) {
    static_assert(pass_floats(RPT, KB) <= kPassFloats, "pass tile larger than the shared tile area");
    const int lp = (int)round_up(a.l + 1, 8);
    const size_t smem = sizeof(Smem);
#define RPCA_BATCH_LAUNCH(CPT)                                                                                    \
    do {                                                                                                          \
        if (cudaFuncSetAttribute(batched_kernel<CPT, RPT, KB>, cudaFuncAttributeMaxDynamicSharedMemorySize,           \
                                 (int)smem) != cudaSuccess)                                                        \
            return RPCA_ERR_CUDA;                                                                                 \
        batched_kernel<CPT, RPT, KB><<<a.grid, kThreads, smem, a.stream>>>(a.items, a.order, a.count, a.l, a.k, a.its, \
                                                                       a.raw, a.seed, a.weights, a.item_status,    \
                                                                       a.active, a.sk1, a.queue, a.slots,          \
                                                                       a.slot_floats, a.max_m);                    \
    } while (0)
    if (lp <= 8) RPCA_BATCH_LAUNCH(1);
    else if (lp <= 16) RPCA_BATCH_LAUNCH(2);
    else if (lp <= 24) RPCA_BATCH_LAUNCH(3);
    else if (lp <= 32) RPCA_BATCH_LAUNCH(4);
    else RPCA_BATCH_LAUNCH(5);
#undef RPCA_BATCH_LAUNCH
    RPCA_CHECK_LAUNCH();
    return RPCA_OK;
}

// instantiated one per translation unit (batched_r2k64.cu, batched_r4k32.cu, ...)
int launch_batched_r2k64(const BatchLaunch &a);
int launch_batched_r4k32(const BatchLaunch &a);
int launch_batched_r8k32(const BatchLaunch &a);

}  // namespace rpca

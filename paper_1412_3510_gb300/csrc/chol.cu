// l x l step of the CholeskyQR renormalisation.
//
// Section 5 renormalises every product with an LU factorisation and the last
// one with a QR factorisation; only the span of the renormalised block enters
// the next product, so any invertible right factor serves.  CholeskyQR takes
// R from the Gram matrix G = Y^T Y = R^T R and forms Q = Y R^-1.  This kernel
// does the l x l part in one CTA: the Cholesky factorisation (FP32, from the
// compensated Gram), a shift of the diagonal when a pivot collapses (the
// shifted CholeskyQR of Fukaya, Kannan, Nakatsukasa, Yamamoto & Yanagisawa,
// SIAM J. Sci. Comput. 42 (2020)), the product with an accumulated triangular
// factor (for B^* = Q2 R2), and the triangular inverse used by the next GEMM.
//
// Cholesky, right-looking and blocked by kNB = 16 (see chol_blocked_kernel): a
// warp factors each diagonal block in registers, the panel to its right is solved
// against it, and the trailing upper triangle is updated in 4 x 4 tiles.
// Inverse: blocked by kNB.  The diagonal blocks are inverted with the factor (lanes
// own columns and sweep the rows bottom-up in lock step); then block rows
// I = nb-2 .. 0 in turn: S = R[I, >I] X[>I, >I], X[I, >I] = -X[I,I] S.
#include "internal.cuh"
#include "gepp.cuh"

namespace rpca {

namespace {

constexpr int kLuThreads = 512;
constexpr int kNB = 16;          // diagonal-block width (16 measured 12 % faster than 32 at l = 102:
                                 // half the shuffles per pivot outweighs twice the panels)

// sum_{t < n} a[t * sa] b[t * sb] with four independent partial sums
__device__ __forceinline__ float dot4(const float *a, int sa, const float *b, int sb, int n) {
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    int t = 0;
    for (; t + 4 <= n; t += 4) {
        s0 = fmaf(a[t * sa], b[t * sb], s0);
        s1 = fmaf(a[(t + 1) * sa], b[(t + 1) * sb], s1);
        s2 = fmaf(a[(t + 2) * sa], b[(t + 2) * sb], s2);
        s3 = fmaf(a[(t + 3) * sa], b[(t + 3) * sb], s3);
    }
    for (; t < n; ++t) s0 = fmaf(a[t * sa], b[t * sb], s0);
    return (s0 + s1) + (s2 + s3);
}

struct CholShared {
    float dorig[RPCA_MAX_L];
    float maxdiag;
    int bad;
};

// skip_flag == 0: R = I (the conditional last round of the final CholeskyQR).
__device__ bool chol_skip(const int *skip_flag, int l, int lp, float *Rinv, const float *Racc_in, float *Racc_out,
                          int *shifted_out) {
    if (!(skip_flag && *skip_flag == 0)) return false;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < lp * lp; e += nt) Rinv[e] = ((e / lp) == (e % lp) && (e / lp) < l) ? 1.f : 0.f;
    if (Racc_out)
        for (int e = tid; e < l * l; e += nt) Racc_out[e] = Racc_in ? Racc_in[e] : ((e / l == e % l) ? 1.f : 0.f);
    if (shifted_out && tid == 0) *shifted_out = 0;
    return true;
}

// the factorization failed even after the shifts: report, R = I
__device__ void chol_fail(bool bad, DevStatus *st, int l, int lp, float *Rinv, float *Racc_out) {
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid == 0) dev_fail(st, bad ? RPCA_ERR_NONFINITE : RPCA_ERR_BREAKDOWN);
    for (int e = tid; e < lp * lp; e += nt) Rinv[e] = ((e / lp) == (e % lp) && (e / lp) < l) ? 1.f : 0.f;
    if (Racc_out)
        for (int e = tid; e < l * l; e += nt) Racc_out[e] = (e / l == e % l) ? 1.f : 0.f;
}

// Racc_out = R Racc_in (or R) from the upper triangle of R (shared memory, row
// stride ld).
__device__ void chol_racc(const float *R, int ld, int l, const float *__restrict__ Racc_in,
                          float *__restrict__ Racc_out) {
    const int tid = threadIdx.x, nt = blockDim.x;
    if (Racc_out) {
        for (int e = tid; e < l * l; e += nt) {
            const int i = e / l, k = e - i * l;
            float v = 0.f;
            if (k >= i)
                v = Racc_in ? dot4(R + i * ld + i, 1, Racc_in + (size_t)i * l + k, l, k - i + 1) : R[i * ld + k];
            Racc_out[e] = v;
        }
    }
}

// Block rows I = nb-2 .. 0 of X = R^-1 in place, the diagonal blocks already
// inverted: S[i][c] = sum_t R[r0+i][t] X[t][c], X[r0+i][c] = -sum_s X[r0+i][r0+s] S[s][c].
// S: kNB x (l - kNB) scratch.  Then Rinv (lp x lp, zero padded).
__device__ void chol_inv_rows(float *R, int ld, float *S, int l, int lp, float *__restrict__ Rinv) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lds = l > kNB ? l - kNB : 1;
    const int nb = (l + kNB - 1) / kNB;
    for (int I = nb - 2; I >= 0; --I) {
        const int r0 = I * kNB, c0 = r0 + kNB;       // block row [r0, c0), columns [c0, l)
        const int w = l - c0;
        for (int e = tid; e < kNB * w; e += nt) {
            const int i = e / w, cc = e - i * w, c = c0 + cc;
            S[i * lds + cc] = dot4(R + (r0 + i) * ld + c0, 1, R + c0 * ld + c, ld, c - c0 + 1);
        }
        __syncthreads();
        for (int e = tid; e < kNB * w; e += nt) {
            const int i = e / w, cc = e - i * w;
            R[(r0 + i) * ld + c0 + cc] = -dot4(R + (r0 + i) * ld + r0 + i, 1, S + i * lds + cc, lds, kNB - i);
        }
        __syncthreads();
    }
    for (int e = tid; e < lp * lp; e += nt) {
        const int i = e / lp, k = e - i * lp;
        Rinv[e] = (i < l && k < l && k >= i) ? R[i * ld + k] : 0.f;
    }
}

// R (upper, shared memory, row stride ld) -> Racc_out = R Racc_in (or R), then R^-1
// in place and Rinv (lp x lp, zero padded).  S: kNB x (l - kNB) scratch.
__device__ void chol_finish(float *R, int ld, float *S, int l, int lp, float *__restrict__ Rinv,
                            const float *__restrict__ Racc_in, float *__restrict__ Racc_out) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31, nwarps = nt >> 5;
    chol_racc(R, ld, l, Racc_in, Racc_out);
    __syncthreads();
    // diagonal blocks, one warp each
    const int nb = (l + kNB - 1) / kNB;
    for (int b = warp; b < nb; b += nwarps) {
        const int b0 = b * kNB, bl = min(kNB, l - b0);
        const int c = b0 + lane;                      // this lane's column
        for (int i = b0 + bl - 1; i >= b0; --i) {
            float x = 0.f;
            if (lane < bl && c >= i)
                x = c == i ? 1.0f / R[i * ld + i]
                           : -dot4(R + i * ld + i + 1, 1, R + (i + 1) * ld + c, ld, c - i) / R[i * ld + i];
            __syncwarp();
            if (lane < bl && c >= i) R[i * ld + c] = x;
            __syncwarp();
        }
    }
    __syncthreads();
    chol_inv_rows(R, ld, S, l, lp, Rinv);
}

__device__ __forceinline__ float next_shift(float shift, int l, float maxdiag) {
    return shift == 0.f ? 16.f * (float)l * 0x1p-24f * fmaxf(maxdiag, 1e-30f) : shift * 100.f;
}

// ---------------------------------------------------------------------------
// Blocked right-looking Cholesky, panels of kNB columns, the whole matrix in shared
// memory (row stride ld = round_up(l, 4), so that rows are 16-byte aligned):
//   1. warp 0 factors the kNB x kNB diagonal block in registers: lane c < kNB holds column
//      c; pivot j is broadcast by shuffles, no CTA barrier inside the block;
//   2. the panel R[J, >J] = X_JJ^T A[J, >J] with the block's inverse X_JJ, in 4 x 4
//      register tiles;
//   3. the trailing update A[>J, >J] -= R[J, >J]^T R[J, >J] in 4 x 4 register tiles
//      of the upper triangle.
// Three barriers per panel instead of one per pivot.
// ---------------------------------------------------------------------------
constexpr int kBlkThreads = 512;
constexpr int kXdLd = kNB + 4;                    // row stride of the diagonal block's inverse

__host__ __device__ __forceinline__ int chol_ld(int l) { return (l + 3) & ~3; }

// Block rows of X = R^-1 (ld a multiple of 4, diagonal blocks already inverted) in
// 2 x 4 register tiles; the strictly lower triangle is cleared first so that every
// sum runs over whole tiles.  S: kNB x (ld - kNB) scratch.  Then Rinv (lp x lp).
constexpr int kTR = 2;                            // rows per register tile of the inverse
__device__ void chol_inv_rows_tiled(float *R, int ld, float *S, int l, int lp, float *__restrict__ Rinv) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31, nwarps = nt >> 5;
    for (int i = warp; i < ld; i += nwarps)
        for (int k = lane; k < i; k += 32) R[i * ld + k] = 0.f;
    __syncthreads();
    const int nb = (l + kNB - 1) / kNB;
    for (int I = nb - 2; I >= 0; --I) {
        const int r0 = I * kNB, c0 = r0 + kNB;
        const int lds = ld - c0, wq = lds / 4;
        // S[i][cc] = sum_{c0 <= t <= c} R[r0+i][t] X[t][c], c = c0 + cc, in kTR x 4 tiles
        // (small tiles: more threads share the triangular work, which is latency-bound)
        for (int q = tid; q < (kNB / kTR) * wq; q += nt) {
            const int iq = q / wq, cq = q - iq * wq;
            const int i0 = r0 + kTR * iq, cc0 = 4 * cq;
            float acc[kTR][4] = {};
            const int tend = c0 + cc0 + 4;
            for (int t = c0; t < tend; ++t) {
                const float4 v = *reinterpret_cast<const float4 *>(R + t * ld + c0 + cc0);
                const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int x = 0; x < kTR; ++x) {
                    const float u = R[(i0 + x) * ld + t];
#pragma unroll
                    for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(u, vv[y], acc[x][y]);
                }
            }
#pragma unroll
            for (int x = 0; x < kTR; ++x)
                *reinterpret_cast<float4 *>(S + (kTR * iq + x) * lds + cc0) =
                    make_float4(acc[x][0], acc[x][1], acc[x][2], acc[x][3]);
        }
        __syncthreads();
        // X[r0+i][c] = -sum_{s >= i} X[r0+i][r0+s] S[s][c - c0]
        for (int q = tid; q < (kNB / kTR) * wq; q += nt) {
            const int iq = q / wq, cq = q - iq * wq;
            const int i0 = kTR * iq, cc0 = 4 * cq;
            float acc[kTR][4] = {};
            for (int sr = i0; sr < kNB; ++sr) {
                const float4 v = *reinterpret_cast<const float4 *>(S + sr * lds + cc0);
                const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int x = 0; x < kTR; ++x) {
                    const float u = R[(r0 + i0 + x) * ld + r0 + sr];
#pragma unroll
                    for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(u, vv[y], acc[x][y]);
                }
            }
#pragma unroll
            for (int x = 0; x < kTR; ++x)
                *reinterpret_cast<float4 *>(R + (r0 + i0 + x) * ld + c0 + cc0) =
                    make_float4(-acc[x][0], -acc[x][1], -acc[x][2], -acc[x][3]);
        }
        __syncthreads();
    }
    for (int i = warp; i < lp; i += nwarps)
        for (int k = lane; k < lp; k += 32) Rinv[(size_t)i * lp + k] = (i < l && k < l && k >= i) ? R[i * ld + k] : 0.f;
}

// A (ld x ld) = G + shift I from the padded Gram (same layout, zero padding), with
// the finiteness of G, its diagonal and its largest diagonal entry in cs (first call).
__device__ void chol_load(const float *__restrict__ G, int l, int ld, float shift, float *A, CholShared &cs,
                          bool first) {
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;
    bool bad = false;
    const int total4 = ld * ld / 4;
    for (int e4 = tid; e4 < total4; e4 += nt) {
        const float4 g = reinterpret_cast<const float4 *>(G)[e4];
        bad |= !(isfinite(g.x) && isfinite(g.y) && isfinite(g.z) && isfinite(g.w));
        reinterpret_cast<float4 *>(A)[e4] = g;
    }
    __syncthreads();
    for (int i = tid; i < l; i += nt) {
        const float v = A[i * ld + i];
        if (first) {
            cs.dorig[i] = v;
            atomicMax(reinterpret_cast<int *>(&cs.maxdiag), __float_as_int(fmaxf(v, 0.f)));
        }
        A[i * ld + i] = v + shift;
    }
    if (first && __any_sync(0xffffffffu, bad) && lane == 0) cs.bad = 1;
}

__global__ void __launch_bounds__(kBlkThreads, 1)
chol_blocked_kernel(const float *__restrict__ G, int l, int lp, float *__restrict__ Rinv,
                    const float *__restrict__ Racc_in, float *__restrict__ Racc_out, DevStatus *__restrict__ st,
                    int *__restrict__ shifted_out, const int *__restrict__ skip_flag) {
    extern __shared__ float4 sm4[];
    float *A = reinterpret_cast<float *>(sm4);
    const int ld = chol_ld(l);
    float *S = A + (size_t)ld * ld;
    __shared__ CholShared cs;
    __shared__ float rdinv[RPCA_MAX_L];           // 1 / R_jj of the factored panels
    __shared__ __align__(16) float Xd[kNB * kXdLd];   // inverse of the current diagonal block
    __shared__ float thr_s[kNB], rdi_s[kNB];
    __shared__ int s_broke;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31;
    if (chol_skip(skip_flag, l, lp, Rinv, Racc_in, Racc_out, shifted_out)) return;
    if (tid == 0) { cs.bad = 0; cs.maxdiag = 0.f; }
    __syncthreads();

    const float tau = 16.f * (float)l * 0x1p-24f;     // a pivot below tau * G_jj has collapsed
    float shift = 0.f;
    bool ok = false;
    for (int attempt = 0; attempt < 4; ++attempt) {
        chol_load(G, l, ld, shift, A, cs, attempt == 0);
        if (tid == 0) s_broke = 0;
        __syncthreads();
        if (cs.bad) break;
        for (int b0 = 0; b0 < l; b0 += kNB) {
            const int bl = min(kNB, l - b0);
            // 1. diagonal block (rows and columns b0 .. b0 + bl - 1): factor, then its
            //    inverse X (column c of X in lane c); R goes to the upper triangle, the
            //    strictly upper part of X transposed to the strictly lower triangle
            if (warp == 0) {
                // Lane c holds column c of the block; the rows of R go through shared memory
                // for the inverse (broadcast reads instead of a shuffle per entry).
                const int c = lane;
                float a[kNB];
#pragma unroll
                for (int r = 0; r < kNB; ++r) a[r] = (r <= c && c < bl) ? A[(b0 + r) * ld + b0 + c] : 0.f;
                if (c < kNB) thr_s[c] = c < bl ? tau * cs.dorig[b0 + c] + 0.5f * shift : 0.f;
                __syncwarp();
                bool fail = false;
                float rd = 1.f;                             // this lane's R_cc
#pragma unroll
                for (int j = 0; j < kNB; ++j) {
                    const float d = __shfl_sync(0xffffffffu, a[j], j);
                    const bool good = j >= bl || (d > thr_s[j] && d > 0.f);
                    fail |= !good;                          // uniform: every lane sees d
                    a[j] *= rsqrtf(j < bl && good ? d : 1.f);   // row j of R: r_jc (lane j: sqrt(d))
                    if (lane == j) rd = a[j];
                    // constant trip counts (r > j resolved at compile time) keep a[] in registers
#pragma unroll
                    for (int r = 0; r < kNB; ++r) {
                        if (r > j) {
                            const float v = __shfl_sync(0xffffffffu, a[j], r);      // r_jr
                            if (c >= r) a[r] = fmaf(-v, a[j], a[r]);
                        }
                    }
                }
                if (fail) {
                    if (lane == 0) s_broke = 1;
                } else {
                    const float rdi = c < bl ? 1.0f / rd : 0.f;
                    // row i of R (entries r_it, t > i, held by lane t) to shared memory (Xd holds
                    // it until X replaces it), and R's upper triangle to A
#pragma unroll
                    for (int r = 0; r < kNB; ++r) {
                        if (c < kNB) Xd[r * kXdLd + c] = (r < c) ? a[r] : 0.f;
                        if (c < bl && r < c) A[(b0 + r) * ld + b0 + c] = a[r];
                    }
                    if (c < kNB) rdi_s[c] = rdi;
                    __syncwarp();
                    // R x = e_c from the bottom: x_i = ([i == c] - sum_{t > i} r_it x_t) / r_ii
                    float x[kNB];
#pragma unroll
                    for (int i = kNB - 1; i >= 0; --i) {
                        float s0 = (i == c) ? 1.f : 0.f, s1 = 0.f;       // two chains of FMAs
#pragma unroll
                        for (int t = 0; t < kNB; ++t) {
                            if (t > i) {
                                const float v = Xd[i * kXdLd + t];
                                if (t & 1) s1 = fmaf(-v, x[t], s1);
                                else s0 = fmaf(-v, x[t], s0);
                            }
                        }
                        x[i] = (s0 + s1) * rdi_s[i];
                    }
                    __syncwarp();                           // every lane has read R from Xd
#pragma unroll
                    for (int r = 0; r < kNB; ++r) {
                        if (c < bl && r < c) A[(b0 + c) * ld + b0 + r] = x[r];
                        if (c < kNB) Xd[r * kXdLd + c] = (c < bl && r <= c) ? x[r] : 0.f;
                    }
                    if (c < bl) {
                        A[(b0 + c) * ld + b0 + c] = rd;
                        rdinv[b0 + c] = rdi;
                    }
                }
            }
            __syncthreads();
            if (s_broke) break;
            const int c0 = b0 + kNB;
            if (c0 >= l) break;
            // 2. panel rows b0 .. b0 + 31, columns c0 .. l - 1 (bl = 32 here):
            //    R[J, c] = X_JJ^T A[J, c]
            //    as 4 x 4 register tiles of X_JJ^T A[J, >J] into S (row stride
            //    lds = ld - c0; padding columns of A are zero, so are those of S)
            const int lds = ld - c0, w = l - c0;
            for (int q = tid; q < (kNB / 4) * (lds / 4); q += nt) {
                const int rq = q / (lds / 4), cq = q - rq * (lds / 4);
                float acc[4][4] = {};
#pragma unroll 8
                for (int t = 0; t < kNB; ++t) {
                    const float4 u = *reinterpret_cast<const float4 *>(Xd + t * kXdLd + 4 * rq);
                    const float4 v = *reinterpret_cast<const float4 *>(A + (b0 + t) * ld + c0 + 4 * cq);
                    const float uu[4] = {u.x, u.y, u.z, u.w}, vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int x = 0; x < 4; ++x)
#pragma unroll
                        for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(uu[x], vv[y], acc[x][y]);
                }
#pragma unroll
                for (int x = 0; x < 4; ++x)
                    *reinterpret_cast<float4 *>(S + (4 * rq + x) * lds + 4 * cq) =
                        make_float4(acc[x][0], acc[x][1], acc[x][2], acc[x][3]);
            }
            __syncthreads();
            for (int e = tid; e < kNB * w; e += nt) {          // the panel back to rows b0 .. b0 + 31
                const int r = e / w, cc = e - r * w;
                A[(b0 + r) * ld + c0 + cc] = S[r * lds + cc];
            }
            const int wq = lds / 4;
            const int ntile = wq * (wq + 1) / 2;
            for (int q = tid; q < ntile; q += nt) {
                int bi = 0, rem = q;
                while (rem >= wq - bi) { rem -= wq - bi; ++bi; }
                const int i0 = c0 + 4 * bi, k0 = c0 + 4 * (bi + rem);
                float acc[4][4];
#pragma unroll
                for (int x = 0; x < 4; ++x)
#pragma unroll
                    for (int y = 0; y < 4; ++y) acc[x][y] = 0.f;
#pragma unroll 8
                for (int t = 0; t < kNB; ++t) {
                    const float4 u = *reinterpret_cast<const float4 *>(S + t * lds + (i0 - c0));
                    const float4 v = *reinterpret_cast<const float4 *>(S + t * lds + (k0 - c0));
                    const float uu[4] = {u.x, u.y, u.z, u.w}, vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int x = 0; x < 4; ++x)
#pragma unroll
                        for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(uu[x], vv[y], acc[x][y]);
                }
#pragma unroll
                for (int x = 0; x < 4; ++x) {
                    float4 *row = reinterpret_cast<float4 *>(A + (i0 + x) * ld + k0);
                    float4 w = *row;
                    w.x -= acc[x][0]; w.y -= acc[x][1]; w.z -= acc[x][2]; w.w -= acc[x][3];
                    *row = w;
                }
            }
            __syncthreads();
        }
        __syncthreads();
        if (!s_broke) { ok = true; break; }
        shift = next_shift(shift, l, cs.maxdiag);
        if (tid == 0) atomicAdd(&st->shifts, 1);
        __syncthreads();
    }
    const bool bad = cs.bad != 0;
    if (shifted_out && tid == 0) *shifted_out = (shift != 0.f || !ok) ? 1 : 0;
    if (!ok) { chol_fail(bad, st, l, lp, Rinv, Racc_out); return; }
    chol_racc(A, ld, l, Racc_in, Racc_out);
    __syncthreads();
    // diagonal blocks of X = R^-1 from the strictly lower triangle (transposed) and rdinv
    for (int e = tid; e < l * kNB; e += nt) {
        const int i = e / kNB, c = (i / kNB) * kNB + (e % kNB);
        if (c < l && c > i) A[i * ld + c] = A[c * ld + i];
        else if (c == i) A[i * ld + i] = rdinv[i];
    }
    __syncthreads();
    chol_inv_rows_tiled(A, ld, S, l, lp, Rinv);
}

// The tall-skinny LU's last step: W = the l pivot rows of Y (ids), partial-pivoting
// LU W = P L U in shared memory, Rinv = U^-1 (lp x lp).  Missing rows (id < 0) enter
// as zero rows; a zero or non-finite pivot (Y rank deficient) is replaced by 1 and
// counted with the shifts, non-finite input is reported.
__global__ void __launch_bounds__(kLuThreads)
lu_final_kernel(const float *__restrict__ Y, int64_t rows, int lp, int l, const int32_t *__restrict__ ids_in,
                float *__restrict__ Rinv, DevStatus *__restrict__ st) {
    extern __shared__ float sm[];
    const int ld = l + 1;
    float *R = sm;
    float *S = sm + (size_t)l * ld;
    __shared__ int ids[RPCA_MAX_L];
    __shared__ GeppScratch g;
    __shared__ int s_bad;
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid == 0) s_bad = 0;
    for (int r = tid; r < l; r += nt) {
        const int id = ids_in[r];
        ids[r] = (id >= 0 && id < rows) ? id : 0x7fffffff;       // present either way
    }
    __syncthreads();
    for (int e = tid; e < l * l; e += nt) {
        const int r = e / l, c = e - r * l;
        const int id = ids[r];
        const float v = id != 0x7fffffff ? Y[(int64_t)id * lp + c] : 0.f;
        if (!isfinite(v)) s_bad = 1;
        R[r * ld + c] = v;
    }
    __syncthreads();
    if (s_bad) {
        if (tid == 0) dev_fail(st, RPCA_ERR_NONFINITE);
        for (int e = tid; e < lp * lp; e += nt) Rinv[e] = ((e / lp) == (e % lp) && (e / lp) < l) ? 1.f : 0.f;
        return;
    }
    gepp_block(R, ld, ids, l, l, g);
    for (int j = tid; j < l; j += nt) {
        const float d = R[j * ld + j];
        if (d == 0.f || !isfinite(d)) {
            R[j * ld + j] = 1.f;
            atomicAdd(&st->shifts, 1);
        }
    }
    __syncthreads();
    chol_finish(R, ld, S, l, lp, Rinv, nullptr, nullptr);
}

}  // namespace

int launch_lu_final(const float *Y, int64_t rows, int lp, int l, const int32_t *ids, float *Rinv, DevStatus *st,
                    cudaStream_t s) {
    const size_t smem = ((size_t)l * (l + 1) + (size_t)kNB * (l > kNB ? l - kNB : 1)) * sizeof(float);
    const size_t smem_max = ((size_t)RPCA_MAX_L * (RPCA_MAX_L + 1) + (size_t)kNB * (RPCA_MAX_L - kNB)) * sizeof(float);
    if (cudaFuncSetAttribute(lu_final_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max) !=
        cudaSuccess)
        return RPCA_ERR_CUDA;
    lu_final_kernel<<<1, kLuThreads, smem, s>>>(Y, rows, lp, l, ids, Rinv, st);
    RPCA_CHECK_LAUNCH();
    return RPCA_OK;
}

int launch_chol_inv(const float *G, int l, int lp, float *Rinv, const float *Racc_in,
                    float *Racc_out, DevStatus *st, cudaStream_t s, int *shifted_out, const int *skip_flag) {
    if (l < 1 || l > RPCA_MAX_L) return RPCA_ERR_INVALID_ARG;
    auto bytes = [](int ll) {
        return ((size_t)chol_ld(ll) * chol_ld(ll) + (size_t)kNB * (chol_ld(ll) > kNB ? chol_ld(ll) - kNB : 4)) *
               sizeof(float);
    };
    if (cudaFuncSetAttribute(chol_blocked_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bytes(RPCA_MAX_L)) != cudaSuccess)
        return RPCA_ERR_CUDA;
    chol_blocked_kernel<<<1, kBlkThreads, bytes(l), s>>>(G, l, lp, Rinv, Racc_in, Racc_out, st, shifted_out,
                                                         skip_flag);
    RPCA_CHECK_LAUNCH();
    return RPCA_OK;
}

}  // namespace rpca

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
// Cholesky, right-looking: step j takes pivot row j, a_jk (k >= j), and updates
// a_ik -= (a_ji / a_jj) a_jk for j < i <= k; row j of R is a_jk / sqrt(a_jj).
//  - l <= 180: every thread keeps a fixed set of upper-triangle entries (the
//    flattened triangle dealt out cyclically) in registers for the whole
//    factorization; the pivot row is double-buffered in shared memory, so a
//    step is one barrier and a few FMAs per thread.
//  - larger l: the entries live in shared memory; warp w updates rows
//    j+1+w, j+33+w, ... with its lanes along the row, one barrier per step.
// Inverse: blocked by 32.  Each warp inverts one 32 x 32 diagonal block
// (lanes own columns and sweep the rows bottom-up in lock step); then block
// rows I = nb-2 .. 0 in turn: S = R[I, >I] X[>I, >I], X[I, >I] = -X[I,I] S.
#include "internal.cuh"
#include "gepp.cuh"

namespace rpca {

namespace {

constexpr int kRegThreads = 512;
constexpr int kBigThreads = 1024;
constexpr int kRegMaxL = 180;          // l (l + 1) / 2 <= 32 entries per thread
constexpr int kNB = 32;

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

// finiteness of G, its diagonal and the largest diagonal entry
__device__ void chol_scan(const double *G, int l, CholShared &cs) {
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid == 0) { cs.bad = 0; cs.maxdiag = 0.f; }
    __syncthreads();
    for (int e = tid; e < l * l; e += nt)
        if (!isfinite(G[e])) cs.bad = 1;
    for (int j = tid; j < l; j += nt) {
        cs.dorig[j] = (float)G[(size_t)j * l + j];
        atomicMax(reinterpret_cast<int *>(&cs.maxdiag), __float_as_int(fmaxf(cs.dorig[j], 0.f)));
    }
    __syncthreads();
}

// the factorization failed even after the shifts: report, R = I
__device__ void chol_fail(bool bad, DevStatus *st, int l, int lp, float *Rinv, float *Racc_out) {
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid == 0) dev_fail(st, bad ? RPCA_ERR_NONFINITE : RPCA_ERR_BREAKDOWN);
    for (int e = tid; e < lp * lp; e += nt) Rinv[e] = ((e / lp) == (e % lp) && (e / lp) < l) ? 1.f : 0.f;
    if (Racc_out)
        for (int e = tid; e < l * l; e += nt) Racc_out[e] = (e / l == e % l) ? 1.f : 0.f;
}

// R (upper, shared memory, row stride ld) -> Racc_out = R Racc_in (or R), then R^-1
// in place and Rinv (lp x lp, zero padded).  S: kNB x (l - kNB) scratch.
__device__ void chol_finish(float *R, int ld, float *S, int l, int lp, float *__restrict__ Rinv,
                            const float *__restrict__ Racc_in, float *__restrict__ Racc_out) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31, nwarps = nt >> 5;
    const int lds = l > kNB ? l - kNB : 1;
    if (Racc_out) {
        for (int e = tid; e < l * l; e += nt) {
            const int i = e / l, k = e - i * l;
            float v = 0.f;
            if (k >= i)
                v = Racc_in ? dot4(R + i * ld + i, 1, Racc_in + (size_t)i * l + k, l, k - i + 1) : R[i * ld + k];
            Racc_out[e] = v;
        }
    }
    __syncthreads();
    // step A: diagonal blocks, one warp each
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
    // step B: block rows bottom-up
    for (int I = nb - 2; I >= 0; --I) {
        const int r0 = I * kNB, c0 = r0 + kNB;       // block row [r0, c0), columns [c0, l)
        const int w = l - c0;
        for (int e = tid; e < kNB * w; e += nt) {    // S[i][c] = sum_{t = c0}^{c} R[r0+i][t] X[t][c]
            const int i = e / w, cc = e - i * w, c = c0 + cc;
            S[i * lds + cc] = dot4(R + (r0 + i) * ld + c0, 1, R + c0 * ld + c, ld, c - c0 + 1);
        }
        __syncthreads();
        for (int e = tid; e < kNB * w; e += nt) {    // X[r0+i][c] = -sum_{s >= i} X[r0+i][r0+s] S[s][c]
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

__device__ __forceinline__ float next_shift(float shift, int l, float maxdiag) {
    return shift == 0.f ? 16.f * (float)l * 0x1p-24f * fmaxf(maxdiag, 1e-30f) : shift * 100.f;
}

// ---------------------------------------------------------------------------
// l <= 180: entries in registers.  Thread t owns entries e = t + s * blockDim.x
// (s < NS) of the upper triangle flattened row by row.
// ---------------------------------------------------------------------------
template <int NS>
__global__ void __launch_bounds__(kRegThreads, 1)
chol_inv_reg_kernel(const double *__restrict__ G, int l, int lp, float *__restrict__ Rinv,
                    const float *__restrict__ Racc_in, float *__restrict__ Racc_out, DevStatus *__restrict__ st,
                    int *__restrict__ shifted_out, const int *__restrict__ skip_flag) {
    extern __shared__ float sm[];
    const int ld = l + 1;
    float *R = sm;                        // l x ld (upper triangle used)
    float *S = sm + (size_t)l * ld;
    __shared__ CholShared cs;
    __shared__ float rowbuf[2][RPCA_MAX_L];
    __shared__ int s_broke;
    const int tid = threadIdx.x, nt = blockDim.x;
    if (chol_skip(skip_flag, l, lp, Rinv, Racc_in, Racc_out, shifted_out)) return;
    chol_scan(G, l, cs);
    const bool bad = cs.bad != 0;

    // this thread's entries: row i, column k (k >= i); unused slots get i = k = l
    int si[NS], sk[NS];
    const int T = l * (l + 1) / 2;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const int e = tid + s * nt;
        int i = l, k = l;
        if (e < T) {
            // rows before i hold off(i) = i (2l - i + 1) / 2 entries; solve off(i) <= e
            const float b = 2.f * l + 1.f;
            i = (int)((b - sqrtf(fmaxf(b * b - 8.f * e, 0.f))) * 0.5f);
            i = max(0, min(i, l - 1));
            while (i + 1 < l && (i + 1) * (2 * l - i) / 2 <= e) ++i;
            while (i > 0 && i * (2 * l - i + 1) / 2 > e) --i;
            k = i + (e - i * (2 * l - i + 1) / 2);
        }
        si[s] = i;
        sk[s] = k;
    }

    const float tau = 16.f * (float)l * 0x1p-24f;     // a pivot below tau * G_jj has collapsed
    float shift = 0.f;
    bool ok = false;
    for (int attempt = 0; attempt < 4 && !bad; ++attempt) {
        float a[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            a[s] = 0.f;
            if (sk[s] < l) {
                a[s] = (float)G[(size_t)si[s] * l + sk[s]];
                if (si[s] == sk[s]) a[s] += shift;
                if (si[s] == 0) rowbuf[0][sk[s]] = a[s];
            }
        }
        if (tid == 0) s_broke = 0;
        __syncthreads();
        for (int j = 0; j < l; ++j) {
            const float *rb = rowbuf[j & 1];
            float *rn = rowbuf[(j + 1) & 1];
            const float d = rb[j];
            if (!(d > tau * cs.dorig[j] + 0.5f * shift) || !(d > 0.f)) {   // uniform: every thread reads d
                if (tid == 0) s_broke = 1;
                break;
            }
            const float inv_d = 1.0f / d;
            const float inv_r = rsqrtf(d);
            for (int t = tid; t < l - j; t += nt) R[j * ld + j + t] = t == 0 ? d * inv_r : rb[j + t] * inv_r;
            // slots run in increasing row order, so the finished ones (row <= j) form a
            // prefix: walk down from the last slot and stop at the first finished one
#pragma unroll
            for (int s = NS - 1; s >= 0; --s) {
                if (si[s] <= j) break;
                if (sk[s] < l) {
                    a[s] = fmaf(-(rb[si[s]] * inv_d), rb[sk[s]], a[s]);
                    if (si[s] == j + 1) rn[sk[s]] = a[s];
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
    if (shifted_out && tid == 0) *shifted_out = (shift != 0.f || !ok) ? 1 : 0;
    if (!ok) { chol_fail(bad, st, l, lp, Rinv, Racc_out); return; }
    chol_finish(R, ld, S, l, lp, Rinv, Racc_in, Racc_out);
}

// ---------------------------------------------------------------------------
// larger l: entries in shared memory.  The scaled pivot row goes to the
// (otherwise unused) lower triangle so that the trailing update of the same step
// can still read the unscaled row; the factor is copied back up at the end.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBigThreads)
chol_inv_big_kernel(const double *__restrict__ G, int l, int lp, float *__restrict__ Rinv,
                    const float *__restrict__ Racc_in, float *__restrict__ Racc_out, DevStatus *__restrict__ st,
                    int *__restrict__ shifted_out, const int *__restrict__ skip_flag) {
    extern __shared__ float sm[];
    const int ld = l + 1;
    float *R = sm;
    float *S = sm + (size_t)l * ld;
    __shared__ CholShared cs;
    __shared__ float rdiag[RPCA_MAX_L];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31, nwarps = nt >> 5;
    if (chol_skip(skip_flag, l, lp, Rinv, Racc_in, Racc_out, shifted_out)) return;
    chol_scan(G, l, cs);
    const bool bad = cs.bad != 0;

    const float tau = 16.f * (float)l * 0x1p-24f;
    float shift = 0.f;
    bool ok = false;
    for (int attempt = 0; attempt < 4 && !bad; ++attempt) {
        for (int e = tid; e < l * l; e += nt) {
            const int i = e / l, k = e - i * l;
            float v = (float)G[e];
            if (i == k) v += shift;
            R[i * ld + k] = v;
        }
        __syncthreads();
        bool broke = false;
        for (int j = 0; j < l; ++j) {
            const float d = R[j * ld + j];
            if (!(d > tau * cs.dorig[j] + 0.5f * shift) || !(d > 0.f)) { broke = true; break; }
            const float inv_d = 1.0f / d;
            const float inv_r = rsqrtf(d);
            for (int i = j + 1 + warp; i < l; i += nwarps) {
                const float rji = R[j * ld + i] * inv_d;
                for (int k = i + lane; k < l; k += 32) R[i * ld + k] = fmaf(-rji, R[j * ld + k], R[i * ld + k]);
            }
            for (int k = j + 1 + tid; k < l; k += nt) R[k * ld + j] = R[j * ld + k] * inv_r;
            if (tid == 0) rdiag[j] = d * inv_r;
            __syncthreads();
        }
        if (!broke) { ok = true; break; }
        __syncthreads();
        shift = next_shift(shift, l, cs.maxdiag);
        if (tid == 0) atomicAdd(&st->shifts, 1);
    }
    if (shifted_out && tid == 0) *shifted_out = (shift != 0.f || !ok) ? 1 : 0;
    if (!ok) { chol_fail(bad, st, l, lp, Rinv, Racc_out); return; }
    for (int e = tid; e < l * l; e += nt) {          // the factor back to the upper triangle
        const int i = e / l, k = e - i * l;
        if (k > i) R[i * ld + k] = R[k * ld + i];
        else if (k == i) R[i * ld + i] = rdiag[i];
    }
    __syncthreads();
    chol_finish(R, ld, S, l, lp, Rinv, Racc_in, Racc_out);
}

// The tall-skinny LU's last step: W = the l pivot rows of Y (ids), partial-pivoting
// LU W = P L U in shared memory, Rinv = U^-1 (lp x lp).  Missing rows (id < 0) enter
// as zero rows; a zero or non-finite pivot (Y rank deficient) is replaced by 1 and
// counted with the shifts, non-finite input is reported.
__global__ void __launch_bounds__(kRegThreads)
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

template <int NS>
int launch_reg(const double *G, int l, int lp, float *Rinv, const float *Racc_in, float *Racc_out, DevStatus *st,
               cudaStream_t s, int *shifted_out, const int *skip_flag, size_t smem, size_t smem_max) {
    if (cudaFuncSetAttribute(chol_inv_reg_kernel<NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max) !=
        cudaSuccess)
        return RPCA_ERR_CUDA;
    chol_inv_reg_kernel<NS><<<1, kRegThreads, smem, s>>>(G, l, lp, Rinv, Racc_in, Racc_out, st, shifted_out,
                                                         skip_flag);
    RPCA_CHECK_LAUNCH();
    return RPCA_OK;
}

}  // namespace

int launch_lu_final(const float *Y, int64_t rows, int lp, int l, const int32_t *ids, float *Rinv, DevStatus *st,
                    cudaStream_t s) {
    const size_t smem = ((size_t)l * (l + 1) + (size_t)kNB * (l > kNB ? l - kNB : 1)) * sizeof(float);
    const size_t smem_max = ((size_t)RPCA_MAX_L * (RPCA_MAX_L + 1) + (size_t)kNB * (RPCA_MAX_L - kNB)) * sizeof(float);
    if (cudaFuncSetAttribute(lu_final_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max) !=
        cudaSuccess)
        return RPCA_ERR_CUDA;
    lu_final_kernel<<<1, kRegThreads, smem, s>>>(Y, rows, lp, l, ids, Rinv, st);
    RPCA_CHECK_LAUNCH();
    return RPCA_OK;
}

int launch_chol_inv(const double *G, int l, int lp, float *Rinv, const float *Racc_in,
                    float *Racc_out, DevStatus *st, cudaStream_t s, int *shifted_out, const int *skip_flag) {
    auto bytes = [](int ll) {
        return ((size_t)ll * (ll + 1) + (size_t)kNB * (ll > kNB ? ll - kNB : 1)) * sizeof(float);
    };
    const size_t smem = bytes(l), smem_max = bytes(RPCA_MAX_L);
    if (l <= kRegMaxL) {
        const int per = (int)cdiv((int64_t)l * (l + 1) / 2, (int64_t)kRegThreads);
#define RPCA_CHOL_REG(NS) launch_reg<NS>(G, l, lp, Rinv, Racc_in, Racc_out, st, s, shifted_out, skip_flag, smem, smem_max)
        if (per <= 2) return RPCA_CHOL_REG(2);
        if (per <= 4) return RPCA_CHOL_REG(4);
        if (per <= 8) return RPCA_CHOL_REG(8);
        if (per <= 12) return RPCA_CHOL_REG(12);
        if (per <= 16) return RPCA_CHOL_REG(16);
        if (per <= 24) return RPCA_CHOL_REG(24);
        return RPCA_CHOL_REG(32);
#undef RPCA_CHOL_REG
    }
    if (cudaFuncSetAttribute(chol_inv_big_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max) !=
        cudaSuccess)
        return RPCA_ERR_CUDA;
    chol_inv_big_kernel<<<1, kBigThreads, smem, s>>>(G, l, lp, Rinv, Racc_in, Racc_out, st, shifted_out, skip_flag);
    RPCA_CHECK_LAUNCH();
    return RPCA_OK;
}

}  // namespace rpca

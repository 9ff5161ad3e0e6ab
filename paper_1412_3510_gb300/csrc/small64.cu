// The l x l steps of the method in FP64 (RPCA_PREC_SMALL_FP64): the Cholesky
// factorisation and triangular inverse of every CholeskyQR renormalisation
// (Section 5 renormalises after every product; any invertible right factor keeps
// the span), the accumulated factor R of B^* = Q2 R, and the SVD of the small
// factor R^T = W Sigma Z^T (Eq. i3).
//
// GB300 issues two FP64 FMAs per clock per SM (a 64th of the FP32 rate), so the
// work is arranged by its shape:
//  * Cholesky, inverse and the product with the accumulated factor: l^3 / 6 FMAs
//    each, one CTA, the upper triangle packed in shared memory (l <= 224 fits:
//    l (l + 1) / 2 doubles).  A pivot below 16 l 2^-24 of its diagonal entry is
//    taken as collapsed and the diagonal shifted, as in the FP32 kernel: that
//    threshold is the noise level of the FP32 Gram matrix the factor comes from,
//    which FP64 arithmetic cannot improve.
//  * SVD: the FP32 one-sided Jacobi of svd.cu gives W, Z and Sigma to FP32
//    accuracy; steps of the iterative refinement of Ogita & Aishima
//    ("Iterative refinement for singular value decomposition based on matrix
//    multiplication", J. Comput. Appl. Math. 369, 2020) take them to FP64
//    accuracy (five steps).  A step is six l x l products in FP64 (spread over all SMs) plus
//    O(l^2) elementwise work:
//      Rm = I - W^T W, Sm = I - Z^T Z, T = W^T (M Z)      (M = R^T)
//      sigma_i = T_ii / (1 - (Rm_ii + Sm_ii) / 2)
//      F_ii = Rm_ii / 2, G_ii = Sm_ii / 2; for i != j, with a = T_ij + Rm_ij sigma_j,
//      b = T_ji + Sm_ij sigma_j: F_ij = (a sigma_j + b sigma_i) / (sigma_j^2 - sigma_i^2),
//      G_ij = (a sigma_i + b sigma_j) / (sigma_j^2 - sigma_i^2)
//      W <- W + W F, Z <- Z + Z G
//    (the first-order conditions of (I + F)^T W^T M Z (I + G) diagonal with W (I + F)
//    and Z (I + G) orthogonal).  For nearly equal sigma_i, sigma_j (relative gap
//    below 2^-20) the pair is left unseparated (F_ij = Rm_ij / 2, G_ij = Sm_ij / 2).
#include "internal.cuh"

#include <algorithm>

namespace rpca {

namespace {

constexpr int kCholThreads = 1024;
// refinement steps: each squares the relative error divided by the relative gap of the
// closest pair; the FP32 Jacobi leaves the left vectors of the smallest values with
// errors up to u sigma_1 / sigma_i, which five steps bring to FP64 level
constexpr int kRefineSteps = 5;

__device__ __forceinline__ int packed_row(int i, int l) { return i * l - (i * (i - 1)) / 2; }

// Warp-strided dot product over t in [t0, t1) of a[t] (packed row i of R, columns t) and
// b(t) = X row t column j (packed), reduced over the warp.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

__global__ void __launch_bounds__(kCholThreads)
chol64_kernel(const float *__restrict__ G, int l, int lp, float *__restrict__ Rinv, const double *__restrict__ Racc_in,
              double *__restrict__ Racc_out, DevStatus *__restrict__ st, int *__restrict__ shifted_out,
              const int *__restrict__ skip_flag) {
    extern __shared__ double P[];                  // packed upper triangle, then a row buffer
    __shared__ double dorig[RPCA_MAX_L];
    __shared__ double s_maxdiag, s_rinv;
    __shared__ int s_fail, s_bad;
    const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, lane = tid & 31, nwarps = nt >> 5;
    const int ldg = gram_ld(l);
    const int np = l * (l + 1) / 2;
    double *row = P + np;                           // l doubles
    if (skip_flag && *skip_flag == 0) {            // R = I
        for (int e = tid; e < lp * lp; e += nt) Rinv[e] = ((e / lp) == (e % lp) && (e / lp) < l) ? 1.f : 0.f;
        if (Racc_out)
            for (int e = tid; e < l * l; e += nt) Racc_out[e] = Racc_in ? Racc_in[e] : ((e / l == e % l) ? 1.0 : 0.0);
        if (shifted_out && tid == 0) *shifted_out = 0;
        return;
    }
    if (tid == 0) { s_maxdiag = 0.0; s_bad = 0; }
    __syncthreads();
    for (int i = tid; i < l; i += nt) {
        const double d = (double)G[(size_t)i * ldg + i];
        dorig[i] = d;
        if (!isfinite(d)) s_bad = 1;
    }
    __syncthreads();
    if (tid == 0)
        for (int i = 0; i < l; ++i) s_maxdiag = fmax(s_maxdiag, dorig[i]);
    const double tau = 16.0 * (double)l * 0x1p-24;
    double shift = 0.0;
    bool ok = false;
    for (int attempt = 0; attempt < 4 && !s_bad; ++attempt) {
        for (int i = warp; i < l; i += nwarps) {
            const int r0 = packed_row(i, l);
            for (int j = i + lane; j < l; j += 32) {
                const float g = G[(size_t)i * ldg + j];
                if (!isfinite(g)) s_bad = 1;
                P[r0 + j - i] = (double)g + (j == i ? shift : 0.0);
            }
        }
        if (tid == 0) s_fail = 0;
        __syncthreads();
        if (s_bad) break;
        // right-looking: pivot k, scale row k, update the trailing upper triangle
        for (int k = 0; k < l; ++k) {
            const int rk = packed_row(k, l);
            if (tid == 0) {
                const double d = P[rk];
                if (!(d > tau * dorig[k] + 0.5 * shift) || !(d > 0.0)) {
                    s_fail = 1;
                } else {
                    const double r = sqrt(d);
                    P[rk] = r;
                    s_rinv = 1.0 / r;
                }
            }
            __syncthreads();
            if (s_fail) break;
            for (int j = k + 1 + tid; j < l; j += nt) P[rk + j - k] *= s_rinv;
            __syncthreads();
            for (int i = k + 1 + warp; i < l; i += nwarps) {
                const double rki = P[rk + i - k];
                const int ri = packed_row(i, l);
                for (int j = i + lane; j < l; j += 32) P[ri + j - i] = fma(-rki, P[rk + j - k], P[ri + j - i]);
            }
            __syncthreads();
        }
        __syncthreads();
        if (!s_fail) { ok = true; break; }
        shift = shift == 0.0 ? tau * fmax(s_maxdiag, 1e-300) : shift * 100.0;
        if (tid == 0) atomicAdd(&st->shifts, 1);
        __syncthreads();
    }
    if (shifted_out && tid == 0) *shifted_out = (shift != 0.0 || !ok) ? 1 : 0;
    if (!ok) {
        if (tid == 0) dev_fail(st, s_bad ? RPCA_ERR_NONFINITE : RPCA_ERR_BREAKDOWN);
        for (int e = tid; e < lp * lp; e += nt) Rinv[e] = ((e / lp) == (e % lp) && (e / lp) < l) ? 1.f : 0.f;
        if (Racc_out)
            for (int e = tid; e < l * l; e += nt) Racc_out[e] = (e / l == e % l) ? 1.0 : 0.0;
        return;
    }
    // Racc_out = R Racc_in (upper x upper), before R is inverted in place
    if (Racc_out) {
        for (int e = warp; e < l * l; e += nwarps) {
            const int i = e / l, kk = e - i * l;
            double v = 0.0;
            if (kk >= i) {
                const int ri = packed_row(i, l);
                if (Racc_in) {
                    for (int t = i + lane; t <= kk; t += 32) v = fma(P[ri + t - i], Racc_in[(size_t)t * l + kk], v);
                    v = warp_sum(v);
                } else {
                    v = P[ri + kk - i];
                }
            }
            if (lane == 0) Racc_out[e] = v;
        }
    }
    __syncthreads();
    // X = R^-1 row by row from the bottom: X_ii = 1 / R_ii, X_ij = -X_ii sum_{i<t<=j} R_it X_tj
    for (int i = l - 1; i >= 0; --i) {
        const int ri = packed_row(i, l);
        const double xii = 1.0 / P[ri];
        for (int j = i + 1 + warp; j < l; j += nwarps) {
            double v = 0.0;
            for (int t = i + 1 + lane; t <= j; t += 32) v = fma(P[ri + t - i], P[packed_row(t, l) + j - t], v);
            v = warp_sum(v);
            if (lane == 0) row[j] = -xii * v;
        }
        __syncthreads();
        for (int j = i + 1 + tid; j < l; j += nt) P[ri + j - i] = row[j];
        if (tid == 0) P[ri] = xii;
        __syncthreads();
    }
    for (int e = tid; e < lp * lp; e += nt) {
        const int i = e / lp, j = e - i * lp;
        Rinv[e] = (i < l && j < l && j >= i) ? (float)P[packed_row(i, l) + j - i] : 0.f;
    }
}

// ---------------------------------------------------------------------------
// the small SVD: FP32 Jacobi, then FP64 refinement
// ---------------------------------------------------------------------------

// C (l x l) = alpha op(A) op(B) + beta C (+ I when add_identity); op = transpose when
// the flag is set.  8 x 8 outputs per CTA, one per thread, FP64.
__global__ void __launch_bounds__(64)
gemm64_kernel(int l, const double *__restrict__ A, bool ta, const double *__restrict__ B, bool tb,
              double *__restrict__ C, double alpha, double beta, bool add_identity) {
    const int i = blockIdx.y * 8 + threadIdx.y, j = blockIdx.x * 8 + threadIdx.x;
    if (i >= l || j >= l) return;
    double v0 = 0.0, v1 = 0.0;
    int t = 0;
    for (; t + 1 < l; t += 2) {
        const double a0 = ta ? A[(size_t)t * l + i] : A[(size_t)i * l + t];
        const double b0 = tb ? B[(size_t)j * l + t] : B[(size_t)t * l + j];
        const double a1 = ta ? A[(size_t)(t + 1) * l + i] : A[(size_t)i * l + t + 1];
        const double b1 = tb ? B[(size_t)j * l + t + 1] : B[(size_t)(t + 1) * l + j];
        v0 = fma(a0, b0, v0);
        v1 = fma(a1, b1, v1);
    }
    if (t < l) {
        const double a0 = ta ? A[(size_t)t * l + i] : A[(size_t)i * l + t];
        const double b0 = tb ? B[(size_t)j * l + t] : B[(size_t)t * l + j];
        v0 = fma(a0, b0, v0);
    }
    double v = alpha * (v0 + v1);
    if (beta != 0.0) v += beta * C[(size_t)i * l + j];
    if (add_identity && i == j) v += 1.0;
    C[(size_t)i * l + j] = v;
}

// From the FP32 Jacobi: W (lp x ldw, columns in descending order), Z (lp x ldw) ->
// W64, Z64 (l x l); M64 = R^T from the FP64 accumulated factor R (l x l, upper).
__global__ void svd64_load_kernel(int l, const float *__restrict__ Wf, const float *__restrict__ Zf, int ldw,
                                  const double *__restrict__ R, double *__restrict__ W64, double *__restrict__ Z64,
                                  double *__restrict__ M64) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < l * l; e += gridDim.x * blockDim.x) {
        const int i = e / l, j = e - i * l;
        W64[e] = (double)Wf[(size_t)i * ldw + j];
        Z64[e] = (double)Zf[(size_t)i * ldw + j];
        M64[e] = R[(size_t)j * l + i];
    }
}

// The refinement's elementwise step: sigma from T, Rm, Sm; F and G (l x l).
__global__ void svd64_update_kernel(int l, const double *__restrict__ T, const double *__restrict__ Rm,
                                    const double *__restrict__ Sm, double *__restrict__ sig, double *__restrict__ F,
                                    double *__restrict__ Gm) {
    extern __shared__ double s_sig[];
    for (int i = threadIdx.x; i < l; i += blockDim.x)
        s_sig[i] = T[(size_t)i * l + i] / (1.0 - 0.5 * (Rm[(size_t)i * l + i] + Sm[(size_t)i * l + i]));
    __syncthreads();
    for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
        const int i = e / l, j = e - i * l;
        double f, g;
        if (i == j) {
            f = 0.5 * Rm[e];
            g = 0.5 * Sm[e];
        } else {
            const double si = s_sig[i], sj = s_sig[j];
            const double den = sj * sj - si * si;
            if (fabs(den) <= 0x1p-20 * fmax(si * si, sj * sj) || den == 0.0) {
                f = 0.5 * Rm[e];
                g = 0.5 * Sm[e];
            } else {
                const double a = T[e] + Rm[e] * sj, b = T[(size_t)j * l + i] + Sm[e] * sj;
                f = (a * sj + b * si) / den;
                g = (a * si + b * sj) / den;
            }
        }
        F[e] = f;
        Gm[e] = g;
    }
    for (int i = threadIdx.x; i < l; i += blockDim.x) sig[i] = s_sig[i];
}

// Outputs: sig (l, descending: a stable sort of the refined values), Wk, Zk (lp x kp,
// the leading k refined columns, FP32, zero padding).
__global__ void svd64_store_kernel(int l, int lp, int k, int kp, const double *__restrict__ sig64,
                                   const double *__restrict__ W64, const double *__restrict__ Z64, float *__restrict__ sig,
                                   float *__restrict__ Wk, float *__restrict__ Zk, double *__restrict__ sig_d,
                                   double *__restrict__ W_d, double *__restrict__ Z_d) {
    __shared__ int order[RPCA_MAX_L];
    for (int j = threadIdx.x; j < l; j += blockDim.x) {
        const double sj = sig64[j];
        int rank = 0;
        for (int i = 0; i < l; ++i) {
            const double si = sig64[i];
            rank += (si > sj) || (si == sj && i < j);
        }
        order[rank] = j;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < l; r += blockDim.x) {
        sig[r] = (float)sig64[order[r]];
        if (sig_d) sig_d[r] = sig64[order[r]];
    }
    if (W_d)
        for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
            const int i = e / l, r = e - i * l;
            W_d[e] = W64[(size_t)i * l + order[r]];
            Z_d[e] = Z64[(size_t)i * l + order[r]];
        }
    for (int e = threadIdx.x; e < lp * kp; e += blockDim.x) {
        const int i = e / kp, r = e - i * kp;
        float w = 0.f, z = 0.f;
        if (i < l && r < k) {
            const int j = order[r];
            w = (float)W64[(size_t)i * l + j];
            z = (float)Z64[(size_t)i * l + j];
        }
        Wk[e] = w;
        Zk[e] = z;
    }
}

// Y += X (count doubles).
__global__ void add64_kernel(int count, const double *__restrict__ X, double *__restrict__ Y) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) Y[e] += X[e];
}

// FP64 l x l R (upper) -> FP32 copy for the Jacobi.
__global__ void narrow_kernel(int count, const double *__restrict__ in, float *__restrict__ out) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) out[e] = (float)in[e];
}

}  // namespace

size_t chol64_smem_bytes(int l) { return ((size_t)l * (l + 1) / 2 + (size_t)l) * sizeof(double); }

int launch_chol64(const float *G, int l, int lp, float *Rinv, const double *Racc_in, double *Racc_out, DevStatus *st,
                  cudaStream_t s, int *shifted_out, const int *skip_flag) {
    if (l < 1 || l > RPCA_MAX_L) return RPCA_ERR_INVALID_ARG;
    if (cudaFuncSetAttribute(chol64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)chol64_smem_bytes(RPCA_MAX_L)) != cudaSuccess)
        return RPCA_ERR_CUDA;
    chol64_kernel<<<1, kCholThreads, chol64_smem_bytes(l), s>>>(G, l, lp, Rinv, Racc_in, Racc_out, st, shifted_out,
                                                               skip_flag);
    RPCA_CHECK_LAUNCH();
    return RPCA_OK;
}

size_t small_svd64_doubles(int l) { return (size_t)10 * l * l + 2 * (size_t)l; }

int launch_small_svd64(const double *R, int l, int lp, int k, int kp, float *Wk, float *Zk, float *sig, float *rot,
                       float *zbuf, int *perm, float *r32, float *wfull, float *zfull, double *scratch, DevStatus *st,
                       cudaStream_t s, double *sig_d, double *W_d, double *Z_d) {
    const int ldw = gram_ld(l);
    const int grid = (int)std::min<int64_t>(cdiv((int64_t)l * l, 256), 64);
    narrow_kernel<<<grid, 256, 0, s>>>(l * l, R, r32);
    RPCA_CHECK_LAUNCH();
    // every singular triplet of R^T in FP32
    RPCA_TRY(launch_small_svd(r32, l, lp, l, ldw, wfull, zfull, sig, rot, zbuf, perm, st, s));
    const size_t ll = (size_t)l * l;
    double *W = scratch, *Z = W + ll, *M = Z + ll, *T = M + ll, *Rm = T + ll, *Sm = Rm + ll, *MZ = Sm + ll,
           *F = MZ + ll, *Gm = F + ll, *tmp = Gm + ll, *sig64 = tmp + ll;
    svd64_load_kernel<<<grid, 256, 0, s>>>(l, wfull, zfull, ldw, R, W, Z, M);
    RPCA_CHECK_LAUNCH();
    const dim3 g8((unsigned)cdiv(l, 8), (unsigned)cdiv(l, 8)), b8(8, 8);
    const size_t usm = (size_t)l * sizeof(double);
    for (int step = 0; step < kRefineSteps; ++step) {
        gemm64_kernel<<<g8, b8, 0, s>>>(l, W, true, W, false, Rm, -1.0, 0.0, true);   // I - W^T W
        RPCA_CHECK_LAUNCH();
        gemm64_kernel<<<g8, b8, 0, s>>>(l, Z, true, Z, false, Sm, -1.0, 0.0, true);   // I - Z^T Z
        RPCA_CHECK_LAUNCH();
        gemm64_kernel<<<g8, b8, 0, s>>>(l, M, false, Z, false, MZ, 1.0, 0.0, false);  // M Z
        RPCA_CHECK_LAUNCH();
        gemm64_kernel<<<g8, b8, 0, s>>>(l, W, true, MZ, false, T, 1.0, 0.0, false);   // W^T M Z
        RPCA_CHECK_LAUNCH();
        svd64_update_kernel<<<1, 1024, usm, s>>>(l, T, Rm, Sm, sig64, F, Gm);
        RPCA_CHECK_LAUNCH();
        // W <- W + W F, Z <- Z + Z G (through tmp: the products read the old W, Z)
        gemm64_kernel<<<g8, b8, 0, s>>>(l, W, false, F, false, tmp, 1.0, 0.0, false);
        RPCA_CHECK_LAUNCH();
        add64_kernel<<<grid, 256, 0, s>>>(l * l, tmp, W);
        RPCA_CHECK_LAUNCH();
        gemm64_kernel<<<g8, b8, 0, s>>>(l, Z, false, Gm, false, tmp, 1.0, 0.0, false);
        RPCA_CHECK_LAUNCH();
        add64_kernel<<<grid, 256, 0, s>>>(l * l, tmp, Z);
        RPCA_CHECK_LAUNCH();
    }
    // the singular values of the refined factors
    gemm64_kernel<<<g8, b8, 0, s>>>(l, W, true, W, false, Rm, -1.0, 0.0, true);
    RPCA_CHECK_LAUNCH();
    gemm64_kernel<<<g8, b8, 0, s>>>(l, Z, true, Z, false, Sm, -1.0, 0.0, true);
    RPCA_CHECK_LAUNCH();
    gemm64_kernel<<<g8, b8, 0, s>>>(l, M, false, Z, false, MZ, 1.0, 0.0, false);
    RPCA_CHECK_LAUNCH();
    gemm64_kernel<<<g8, b8, 0, s>>>(l, W, true, MZ, false, T, 1.0, 0.0, false);
    RPCA_CHECK_LAUNCH();
    svd64_update_kernel<<<1, 1024, usm, s>>>(l, T, Rm, Sm, sig64, F, Gm);
    RPCA_CHECK_LAUNCH();
    svd64_store_kernel<<<1, 1024, 0, s>>>(l, lp, k, kp, sig64, W, Z, sig, Wk, Zk, sig_d, W_d, Z_d);
    RPCA_CHECK_LAUNCH();
    return RPCA_OK;
}

}  // namespace rpca

namespace {

// M (l x l, row-major) -> R = M^T, the layout the small-SVD kernels take (they factor R^T).
__global__ void transpose64_kernel(int l, const double *__restrict__ M, double *__restrict__ R) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < l * l; e += gridDim.x * blockDim.x) {
        const int i = e / l, j = e - i * l;
        R[(size_t)j * l + i] = M[e];
    }
}

struct SvdPlan {
    size_t status, R, rot, zbuf, perm, r32, wfull, zfull, wk, zk, sig, scratch, total;
};

SvdPlan svd_plan(int l) {
    auto a256 = [](size_t x) { return (x + 255) & ~(size_t)255; };
    SvdPlan P;
    const int lp = rpca::padded_l(l), ldw = rpca::gram_ld(l);
    size_t off = 0;
    auto take = [&](size_t b) { const size_t o = off; off = a256(off + b); return o; };
    P.status = take(sizeof(rpca::DevStatus));
    P.R = take((size_t)l * l * 8);
    P.rot = take(rpca::small_svd_rot_floats(l) * 4);
    P.zbuf = take(256);
    P.perm = take((size_t)lp * 4);
    P.r32 = take((size_t)l * l * 4);
    P.wfull = take((size_t)lp * ldw * 4);
    P.zfull = take((size_t)lp * ldw * 4);
    P.wk = take((size_t)lp * ldw * 4);
    P.zk = take((size_t)lp * ldw * 4);
    P.sig = take((size_t)lp * 4);
    P.scratch = take(rpca::small_svd64_doubles(l) * 8);
    P.total = off;
    return P;
}

}  // namespace

extern "C" size_t rpca_small_svd_workspace_size(int32_t l) {
    if (l < 1 || l > RPCA_MAX_L) return 0;
    return svd_plan(l).total;
}

extern "C" int rpca_small_svd(const double *M, int32_t l, double *S, double *W, double *Z, void *ws, size_t ws_bytes,
                              rpca_stream_t stream) {
    if (!M || !S || !W || !Z || l < 1 || l > RPCA_MAX_L) return RPCA_ERR_INVALID_ARG;
    const SvdPlan P = svd_plan(l);
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0 || ws_bytes < P.total) return RPCA_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    char *b = reinterpret_cast<char *>(ws);
    auto *st = reinterpret_cast<rpca::DevStatus *>(b + P.status);
    if (cudaMemsetAsync(st, 0, sizeof(rpca::DevStatus), s) != cudaSuccess) return RPCA_ERR_CUDA;
    double *R = reinterpret_cast<double *>(b + P.R);
    transpose64_kernel<<<(unsigned)std::min<int64_t>(rpca::cdiv((int64_t)l * l, 256), 64), 256, 0, s>>>(l, M, R);
    RPCA_CHECK_LAUNCH();
    const int lp = rpca::padded_l(l), ldw = rpca::gram_ld(l);
    return rpca::launch_small_svd64(R, l, lp, l, ldw, reinterpret_cast<float *>(b + P.wk),
                                    reinterpret_cast<float *>(b + P.zk), reinterpret_cast<float *>(b + P.sig),
                                    reinterpret_cast<float *>(b + P.rot), reinterpret_cast<float *>(b + P.zbuf),
                                    reinterpret_cast<int *>(b + P.perm), reinterpret_cast<float *>(b + P.r32),
                                    reinterpret_cast<float *>(b + P.wfull), reinterpret_cast<float *>(b + P.zfull),
                                    reinterpret_cast<double *>(b + P.scratch), st, s, S, W, Z);
}

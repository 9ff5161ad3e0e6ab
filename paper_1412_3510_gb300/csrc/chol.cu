// l x l step of the CholeskyQR renormalisation.
//
// Section 5 renormalises every product with an LU factorisation and the last
// one with a QR factorisation; only the span of the renormalised block enters
// the next product, so any invertible right factor serves.  CholeskyQR takes
// R from the Gram matrix G = Y^T Y = R^T R and forms Q = Y R^-1.  This kernel
// does the l x l part in one CTA: the Cholesky factorisation (FP32, from the
// FP64-accumulated Gram), a shift of the diagonal when a pivot collapses (the
// shifted CholeskyQR of Fukaya, Kannan, Nakatsukasa, Yamamoto & Yanagisawa,
// SIAM J. Sci. Comput. 42 (2020)), the product with an accumulated triangular
// factor (for B^* = Q2 R2), and the triangular inverse used by the next GEMM.
#include "internal.cuh"

namespace rpca {

namespace {

constexpr int kCholThreads = 1024;

__global__ void __launch_bounds__(kCholThreads)
chol_inv_kernel(const double *__restrict__ G, int l, int lp, float *__restrict__ Rinv,
                const float *__restrict__ Racc_in, float *__restrict__ Racc_out,
                DevStatus *__restrict__ st) {
    extern __shared__ float sm[];
    const int ld = l + 1;
    float *R = sm;                    // l x ld
    float *col = sm + (size_t)l * ld; // l floats
    __shared__ float dorig[RPCA_MAX_L];
    __shared__ float s_maxdiag;
    __shared__ int s_bad;
    const int tid = threadIdx.x, nt = blockDim.x;

    if (tid == 0) { s_bad = 0; s_maxdiag = 0.f; }
    __syncthreads();
    for (int e = tid; e < l * l; e += nt) {
        const double g = G[e];
        if (!isfinite(g)) atomicOr(&s_bad, 1);
    }
    for (int j = tid; j < l; j += nt) {
        dorig[j] = (float)G[(size_t)j * l + j];
        atomicMax(reinterpret_cast<int *>(&s_maxdiag), __float_as_int(fmaxf(dorig[j], 0.f)));
    }
    __syncthreads();
    const bool bad = s_bad != 0;
    const float maxdiag = s_maxdiag;

    // tolerance for a collapsed pivot, and the shift of the first retry
    const float eps = 0x1p-24f;
    const float tau = 16.f * (float)l * eps;
    float shift = 0.f;
    bool ok = false;
    for (int attempt = 0; attempt < 4 && !bad; ++attempt) {
        for (int e = tid; e < l * l; e += nt) {
            const int i = e / l, k = e % l;
            float v = (float)G[e];
            if (i == k) v += shift;
            R[i * ld + k] = v;
        }
        __syncthreads();
        bool broke = false;
        for (int j = 0; j < l; ++j) {
            const float d = R[j * ld + j];
            if (!(d > tau * dorig[j] + shift * 0.5f) || !(d > 0.f)) { broke = true; break; }
            const float rjj = sqrtf(d);
            const float inv = 1.0f / rjj;
            __syncthreads();                         // everyone has read d
            for (int k = j + 1 + tid; k < l; k += nt) R[j * ld + k] *= inv;
            if (tid == 0) R[j * ld + j] = rjj;
            __syncthreads();
            const int rem = l - j - 1;
            for (int e = tid; e < rem * rem; e += nt) {
                const int i = j + 1 + e / rem, k = j + 1 + e % rem;
                if (k >= i) R[i * ld + k] -= R[j * ld + i] * R[j * ld + k];
            }
            __syncthreads();
        }
        if (!broke) { ok = true; break; }
        __syncthreads();
        shift = (shift == 0.f) ? 16.f * (float)l * eps * fmaxf(maxdiag, 1e-30f) : shift * 100.f;
        if (tid == 0) atomicAdd(&st->shifts, 1);
    }

    if (!ok) {
        if (tid == 0) dev_fail(st, bad ? RPCA_ERR_NONFINITE : RPCA_ERR_BREAKDOWN);
        for (int e = tid; e < lp * lp; e += nt) Rinv[e] = ((e / lp) == (e % lp) && (e / lp) < l) ? 1.f : 0.f;
        if (Racc_out)
            for (int e = tid; e < l * l; e += nt) Racc_out[e] = (e / l == e % l) ? 1.f : 0.f;
        return;
    }

    // Racc_out = R * Racc_in (both upper triangular), or R itself.
    if (Racc_out) {
        for (int e = tid; e < l * l; e += nt) {
            const int i = e / l, k = e % l;
            float v = 0.f;
            if (k >= i) {
                if (Racc_in) {
                    for (int t = i; t <= k; ++t) v = fmaf(R[i * ld + t], Racc_in[(size_t)t * l + k], v);
                } else {
                    v = R[i * ld + k];
                }
            }
            Racc_out[e] = v;
        }
    }
    __syncthreads();

    // In-place inverse X = R^-1, one column k at a time:
    // X[k][k] = 1 / R[k][k];  X[i][k] = -(sum_{t=i}^{k-1} X[i][t] R[t][k]) / R[k][k], i < k.
    // Columns t < k of X already overwrite those of R; column k of R is copied first.
    const int lane4 = tid & 3;
    const int row = tid >> 2;            // 4 threads per row, rows 0..255
    for (int k = 0; k < l; ++k) {
        for (int t = tid; t <= k; t += nt) col[t] = R[t * ld + k];
        __syncthreads();
        const float rkk_inv = 1.0f / col[k];
        float v = 0.f;
        if (row < k) {
            for (int t = row + lane4; t < k; t += 4) v = fmaf(R[row * ld + t], col[t], v);
        }
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        v += __shfl_xor_sync(0xffffffffu, v, 2);
        __syncthreads();
        if (lane4 == 0) {
            if (row < k) R[row * ld + k] = -v * rkk_inv;
            else if (row == k) R[row * ld + k] = rkk_inv;
        }
        __syncthreads();
    }

    for (int e = tid; e < lp * lp; e += nt) {
        const int i = e / lp, k = e % lp;
        Rinv[e] = (i < l && k < l && k >= i) ? R[i * ld + k] : 0.f;
    }
}

}  // namespace

int launch_chol_inv(const double *G, int l, int lp, float *Rinv, const float *Racc_in,
                    float *Racc_out, DevStatus *st, cudaStream_t s) {
    const size_t smem = ((size_t)l * (l + 1) + l) * sizeof(float);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(chol_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(((size_t)RPCA_MAX_L * (RPCA_MAX_L + 1) + RPCA_MAX_L) * sizeof(float)));
        attr_set = true;
    }
    chol_inv_kernel<<<1, kCholThreads, smem, s>>>(G, l, lp, Rinv, Racc_in, Racc_out, st);
    RPCA_CHECK_LAUNCH();
    return RPCA_OK;
}

}  // namespace rpca

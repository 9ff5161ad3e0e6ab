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
//
// Cholesky: right-looking, one barrier per column; warp w updates rows
// j+1+w, j+33+w, ... of the trailing upper triangle with its lanes running
// along the row.  The scaled pivot row is written to the (otherwise unused)
// lower triangle, so the trailing update of the same step can still read the
// unscaled row; the factor is copied back up at the end.
// Inverse: blocked by 32.  Each warp inverts one 32 x 32 diagonal block
// (lanes own columns and sweep the rows bottom-up in lock step); then block
// rows I = nb-2 .. 0 in turn: S = R[I, >I] X[>I, >I], X[I, >I] = -X[I,I] S.
#include "internal.cuh"

namespace rpca {

namespace {

constexpr int kCholThreads = 1024;
constexpr int kNB = 32;

__global__ void __launch_bounds__(kCholThreads)
chol_inv_kernel(const double *__restrict__ G, int l, int lp, float *__restrict__ Rinv,
                const float *__restrict__ Racc_in, float *__restrict__ Racc_out,
                DevStatus *__restrict__ st, int *__restrict__ shifted_out, const int *__restrict__ skip_flag) {
    extern __shared__ float sm[];
    const int ld = l + 1;
    float *R = sm;                        // l x ld
    float *S = sm + (size_t)l * ld;       // kNB x (l - kNB) scratch for the blocked inverse
    const int lds = l > kNB ? l - kNB : 1;
    __shared__ float dorig[RPCA_MAX_L];
    __shared__ float rdiag[RPCA_MAX_L];   // diagonal of the factor (R[j][j] still holds pivots)
    __shared__ float s_maxdiag;
    __shared__ int s_bad;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31, nwarps = nt >> 5;

    if (skip_flag && *skip_flag == 0) {                 // R = I
        for (int e = tid; e < lp * lp; e += nt) Rinv[e] = ((e / lp) == (e % lp) && (e / lp) < l) ? 1.f : 0.f;
        if (Racc_out)
            for (int e = tid; e < l * l; e += nt)
                Racc_out[e] = Racc_in ? Racc_in[e] : ((e / l == e % l) ? 1.f : 0.f);
        if (shifted_out && tid == 0) *shifted_out = 0;
        return;
    }
    if (tid == 0) { s_bad = 0; s_maxdiag = 0.f; }
    __syncthreads();
    for (int e = tid; e < l * l; e += nt)
        if (!isfinite(G[e])) s_bad = 1;
    for (int j = tid; j < l; j += nt) {
        dorig[j] = (float)G[(size_t)j * l + j];
        atomicMax(reinterpret_cast<int *>(&s_maxdiag), __float_as_int(fmaxf(dorig[j], 0.f)));
    }
    __syncthreads();
    const bool bad = s_bad != 0;
    const float maxdiag = s_maxdiag;

    const float eps = 0x1p-24f;
    const float tau = 16.f * (float)l * eps;     // a pivot below tau * G_jj has collapsed
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
            if (!(d > tau * dorig[j] + 0.5f * shift) || !(d > 0.f)) { broke = true; break; }
            const float inv_d = 1.0f / d;
            const float inv_r = rsqrtf(d);
            // trailing update with the unscaled row j: R[i][k] -= R[j][i] R[j][k] / d, j < i <= k
            for (int i = j + 1 + warp; i < l; i += nwarps) {
                const float rji = R[j * ld + i] * inv_d;
                for (int k = i + lane; k < l; k += 32) R[i * ld + k] = fmaf(-rji, R[j * ld + k], R[i * ld + k]);
            }
            // the scaled row j goes to column j of the lower triangle
            for (int k = j + 1 + tid; k < l; k += nt) R[k * ld + j] = R[j * ld + k] * inv_r;
            if (tid == 0) rdiag[j] = d * inv_r;
            __syncthreads();
        }
        if (!broke) { ok = true; break; }
        __syncthreads();
        shift = (shift == 0.f) ? 16.f * (float)l * eps * fmaxf(maxdiag, 1e-30f) : shift * 100.f;
        if (tid == 0) atomicAdd(&st->shifts, 1);
    }
    if (shifted_out && tid == 0) *shifted_out = (shift != 0.f || !ok) ? 1 : 0;

    if (!ok) {
        if (tid == 0) dev_fail(st, bad ? RPCA_ERR_NONFINITE : RPCA_ERR_BREAKDOWN);
        for (int e = tid; e < lp * lp; e += nt) Rinv[e] = ((e / lp) == (e % lp) && (e / lp) < l) ? 1.f : 0.f;
        if (Racc_out)
            for (int e = tid; e < l * l; e += nt) Racc_out[e] = (e / l == e % l) ? 1.f : 0.f;
        return;
    }
    // copy the factor back to the upper triangle
    for (int e = tid; e < l * l; e += nt) {
        const int i = e / l, k = e - i * l;
        if (k > i) R[i * ld + k] = R[k * ld + i];
        else if (k == i) R[i * ld + i] = rdiag[i];
    }
    __syncthreads();

    // Racc_out = R * Racc_in (both upper triangular), or R itself.
    if (Racc_out) {
        for (int e = tid; e < l * l; e += nt) {
            const int i = e / l, k = e - i * l;
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

    // ---- inverse, step A: diagonal blocks, one warp each ----
    const int nb = (l + kNB - 1) / kNB;
    for (int b = warp; b < nb; b += nwarps) {
        const int b0 = b * kNB, bl = min(kNB, l - b0);
        const int c = b0 + lane;                      // this lane's column
        for (int i = b0 + bl - 1; i >= b0; --i) {
            float x = 0.f;
            if (lane < bl && c >= i) {
                if (c == i) {
                    x = 1.0f / R[i * ld + i];
                } else {
                    float s = 0.f;
                    for (int t = i + 1; t <= c; ++t) s = fmaf(R[i * ld + t], R[t * ld + c], s);
                    x = -s / R[i * ld + i];
                }
            }
            __syncwarp();
            if (lane < bl && c >= i) R[i * ld + c] = x;
            __syncwarp();
        }
    }
    __syncthreads();

    // ---- step B: block rows bottom-up ----
    for (int I = nb - 2; I >= 0; --I) {
        const int r0 = I * kNB, c0 = r0 + kNB;       // block row [r0, c0), columns [c0, l)
        const int w = l - c0;
        // S[i][c] = sum_{t = c0}^{c} R[r0+i][t] X[t][c]
        for (int e = tid; e < kNB * w; e += nt) {
            const int i = e / w, cc = e - i * w, c = c0 + cc;
            float s = 0.f;
            for (int t = c0; t <= c; ++t) s = fmaf(R[(r0 + i) * ld + t], R[t * ld + c], s);
            S[i * lds + cc] = s;
        }
        __syncthreads();
        // X[r0+i][c] = - sum_{s = i}^{kNB-1} X[r0+i][r0+s] S[s][c]
        for (int e = tid; e < kNB * w; e += nt) {
            const int i = e / w, cc = e - i * w;
            float v = 0.f;
            for (int s2 = i; s2 < kNB; ++s2) v = fmaf(R[(r0 + i) * ld + r0 + s2], S[s2 * lds + cc], v);
            R[(r0 + i) * ld + c0 + cc] = -v;
        }
        __syncthreads();
    }

    for (int e = tid; e < lp * lp; e += nt) {
        const int i = e / lp, k = e - i * lp;
        Rinv[e] = (i < l && k < l && k >= i) ? R[i * ld + k] : 0.f;
    }
}

}  // namespace

int launch_chol_inv(const double *G, int l, int lp, float *Rinv, const float *Racc_in,
                    float *Racc_out, DevStatus *st, cudaStream_t s, int *shifted_out, const int *skip_flag) {
    const size_t smem = ((size_t)l * (l + 1) + (size_t)kNB * (l > kNB ? l - kNB : 1)) * sizeof(float);
    if (cudaFuncSetAttribute(chol_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(((size_t)RPCA_MAX_L * (RPCA_MAX_L + 1) + (size_t)kNB * (RPCA_MAX_L - kNB)) *
                                   sizeof(float))) != cudaSuccess)
        return RPCA_ERR_CUDA;
    chol_inv_kernel<<<1, kCholThreads, smem, s>>>(G, l, lp, Rinv, Racc_in, Racc_out, st, shifted_out, skip_flag);
    RPCA_CHECK_LAUNCH();
    return RPCA_OK;
}

}  // namespace rpca

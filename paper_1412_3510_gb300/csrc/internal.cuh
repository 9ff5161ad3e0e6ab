// Internal declarations shared by the translation units of librpca.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include <algorithm>

#include "rpca.h"

namespace rpca {

// ---------------------------------------------------------------------------
// device status word (first 256 bytes of every workspace)
// ---------------------------------------------------------------------------
struct DevStatus {
    int32_t status;        // 0, or the most severe (most negative) error code
    int32_t flags;         // bit 0: fell back (informative)
    int32_t shifts;        // number of shifted Cholesky factorisations
    int32_t jacobi_sweeps; // sweeps used by the last small SVD
    int32_t jacobi_unconverged;
    int32_t timeouts;
    int32_t pad[58];
};
static_assert(sizeof(DevStatus) == 256, "status block is 256 bytes");

__device__ __forceinline__ void dev_fail(DevStatus *st, int code) {
    atomicMin(&st->status, code);
}

// ---------------------------------------------------------------------------
// launch accounting
// ---------------------------------------------------------------------------
void count_launch();
int check_launch();   // RPCA_OK or RPCA_ERR_CUDA after a <<<>>> launch

#define RPCA_CHECK_LAUNCH()                                  \
    do {                                                     \
        rpca::count_launch();                                \
        int _e = rpca::check_launch();                       \
        if (_e != RPCA_OK) return _e;                        \
    } while (0)

#define RPCA_TRY(expr)                                       \
    do {                                                     \
        int _e = (expr);                                     \
        if (_e < 0) return _e;                               \
    } while (0)

__host__ __device__ inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ inline int64_t round_up(int64_t a, int64_t b) { return cdiv(a, b) * b; }

// Padded sketch width: at least one spare column (the ones column that
// carries the column sums of A through the adjoint products), multiple of 8.
static inline int padded_l(int l) { return (int)round_up(l + 1, 8); }

// The precision of the passes over A, and the FP64 modifier of the l x l work.
static inline int pass_precision(int p) { return p & ~RPCA_PREC_SMALL_FP64; }
static inline bool small_fp64(int p) { return (p & RPCA_PREC_SMALL_FP64) != 0; }

int num_sms();

// ---------------------------------------------------------------------------
// launchers (each returns an rpca_status)
// ---------------------------------------------------------------------------

// Omega: n x l Gaussian (optionally scaled by row weights d[i]), written into
// out (leading dimension ldo).  Columns [l, ldo) are not touched.
int launch_omega(int64_t n, int l, uint64_t seed, uint64_t stream_id, const float *weights,
                 float *out, int64_t ldo, cudaStream_t s);

// C[M x N] (ldc) = op(A) B over the K range split into `splits` slices;
// slice z writes C + z * split_stride.  op(A) = A (A is M x K, lda) when
// !trans_a, and A^T (A stored K x M, lda) when trans_a.  B is K x N (ldb).
// When copy_flag is given and *copy_flag == 0 (read on the device), the
// kernel copies C = A (non-transposed, M x N) instead of multiplying.  bias
// (N values, non-transposed and unsplit only): C = A B - 1 bias, Section 5's
// implicit centring with bias = c B.
int launch_sgemm(bool trans_a, int64_t M, int64_t N, int64_t K, const float *A, int64_t lda,
                 const float *B, int64_t ldb, float *C, int64_t ldc, int splits,
                 int64_t split_stride, cudaStream_t s, const int *copy_flag = nullptr,
                 const float *bias = nullptr);

// Partial Grams part[s] (lp x lp) = Y[chunk s]^T Y[chunk s] of a row-major Y
// (rows x lp, ld = lp); skipped entirely when *skip_flag == 0.
int launch_gram(const float *Y, int64_t rows, int lp, float *part, int splits, const int *skip_flag,
                cudaStream_t s);
int gram_splits(int64_t rows, int lp);
// tall-skinny LU with tournament pivoting (renorm = LU): the l pivot rows of Y, then
// Rinv = U^-1 from the LU of those rows
size_t tslu_ids_bytes(int64_t rows, int l);
bool tslu_supported(int l);
int launch_tslu_select(const float *Y, int64_t rows, int lp, int l, int32_t *buf0, int32_t *buf1,
                       const int32_t **winner, cudaStream_t s);
int launch_lu_final(const float *Y, int64_t rows, int lp, int l, const int32_t *ids, float *Rinv, DevStatus *st,
                    cudaStream_t s);

// Number of K slices launch_sgemm should use so that the grid fills the GPU.
int choose_splits(int64_t M, int64_t N, int64_t K);

// Column sums of the first l columns of Y (rows x ld), partial per chunk of
// rows: part[chunk * l + c].  Returns the number of chunks via *nchunks.
int launch_colsum_partial(const float *Y, int64_t rows, int l, int64_t ld, float *part,
                          int *nchunks, cudaStream_t s);
int colsum_chunks(int64_t rows);

// Y[i][c] -= mean_c for c < l (mean from the partials), Y[i][c] = 0 for l <= c < ld.
int launch_center(float *Y, int64_t rows, int l, int64_t ld, const float *part, int nchunks,
                  cudaStream_t s);

// Finish a renormalised tall block: Q[:, l] = ones_value, Q[:, l+1:ld) = 0;
// when part != NULL also write per-chunk column sums of Q[:, :l].
int launch_finalize(float *Q, int64_t rows, int l, int64_t ld, float ones_value, float *part,
                    cudaStream_t s);

// Row stride of the reduced Gram matrix: l rounded up to a multiple of 4.
__host__ __device__ inline int gram_ld(int l) { return (l + 3) & ~3; }
// G (FP32, gram_ld(l) x gram_ld(l), zero padding) = compensated sum over splits of the
// FP32 partial Grams part[s] (lp x lp).
int launch_gram_reduce(const float *part, int splits, int l, int lp, float *G, cudaStream_t s,
                       const int *skip_flag = nullptr);

// X = sum_s part[s] (rows x lp); when centring, X[:, c] -= (X[:, l] / m) * qsum[c]
// with qsum from the column-sum partials of Q; padding columns zeroed.  cvec
// (optional, centring only): the column means of A, c[j] = X[j][l] / m.
int launch_adjoint_reduce(const float *part, int splits, int64_t rows, int l, int lp, float *X,
                          int centre, double m, const float *qpart, int qchunks, cudaStream_t s,
                          float *cvec = nullptr);

// bias[j] = sum_i c[i] X[i][j] for j < l, 0 for l <= j < lp (c: n values, X: n x lp):
// the row vector c X of Section 5's implicit centring A*X - ones(m,1)*(c*X).  part:
// centring_parts(n) x lp floats of scratch.
int centring_parts(int64_t n);
int launch_centring_row(const float *c, const float *X, int64_t n, int l, int lp, float *part, float *bias,
                        cudaStream_t s);

// One CTA: Cholesky G = R^T R in FP32 (shifted on breakdown), Rinv (lp x lp,
// zero padded) = R^-1; optionally Racc_out = R * Racc_in (l x l, upper).
// shifted_out (optional) receives 1 when the diagonal had to be shifted.
// When skip_flag is given and *skip_flag == 0, R = I: Rinv = I and
// Racc_out = Racc_in.
int launch_chol_inv(const float *G, int l, int lp, float *Rinv, const float *Racc_in,
                    float *Racc_out, DevStatus *st, cudaStream_t s, int *shifted_out = nullptr,
                    const int *skip_flag = nullptr);

// The same factorisation in FP64 (RPCA_PREC_SMALL_FP64): Racc_in / Racc_out are l x l
// FP64; Rinv is FP32 for the tall products.
int launch_chol64(const float *G, int l, int lp, float *Rinv, const double *Racc_in, double *Racc_out, DevStatus *st,
                  cudaStream_t s, int *shifted_out = nullptr, const int *skip_flag = nullptr);

// Small SVD of R^T to FP64 accuracy: the FP32 Jacobi below on an FP32 copy of R, then
// FP64 refinement.  r32 (l x l floats), wfull and zfull (lp x gram_ld(l) floats each) and
// scratch (small_svd64_doubles(l) doubles) are workspace; outputs as launch_small_svd.
size_t small_svd64_doubles(int l);
int launch_small_svd64(const double *R, int l, int lp, int k, int kp, float *Wk, float *Zk, float *sig, float *rot,
                       float *zbuf, int *perm, float *r32, float *wfull, float *zfull, double *scratch, DevStatus *st,
                       cudaStream_t s, double *sig_d = nullptr, double *W_d = nullptr, double *Z_d = nullptr);

// Small SVD of R^T (R = Racc, l x l upper): writes Wk (lp x kp, U-side
// factors, k leading left singular vectors of R^T), sig (l, descending) and
// Zk (lp x kp, V-side).  rot/zbuf are scratch.
int launch_small_svd(const float *R, int l, int lp, int k, int kp, float *Wk, float *Zk,
                     float *sig, float *rot, float *zbuf, int *perm, DevStatus *st, cudaStream_t s);
size_t small_svd_rot_floats(int l);

// Sign convention and singular values: for r < k, flip V[:, r] so that its
// largest-magnitude entry is positive, scale Wk's column r by the same sign,
// and write S[r] = sig[r].
int launch_sign_fix(float *V, int64_t n, int64_t ldv, int k, float *Wk, int lp, int kp,
                    const float *sig, float *S, cudaStream_t s);

// Residual estimator kernels (power method on E = A_c - U S V^T).
int launch_fill(float *p, int64_t count, float value, cudaStream_t s);

}  // namespace rpca

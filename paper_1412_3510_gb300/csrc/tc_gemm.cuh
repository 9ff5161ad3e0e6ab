// tcgen05 split-BF16 pass kernels (see tc_gemm.cu).
#pragma once

#include <cuda_bf16.h>

#include "internal.cuh"

namespace rpca {

int tc_n(int lp);                                     // MMA N for a padded width lp
int tc_bk(int lp);                                    // K per pipeline stage
bool tc_supported(const float *A, int64_t lda, int lp);
size_t tc_split_bytes(int64_t rows, int lp);          // pre-split block operand size
int tc_adjoint_splits(int64_t n, int64_t m, int lp);

// FP32 block P (rows x lp) -> BF16 hi/lo per stage in the MMA's K-major layout.
int launch_tc_split(const float *P, int64_t rows, int lp, __nv_bfloat16 *out, cudaStream_t s);
// Y (m x lp) = A X, X given pre-split; with bias (lp values), Y = A X - 1 bias.
// tail_part (optional, tc_apply_tail_bytes(lp) bytes): room for the K pieces of the
// last partial wave of row tiles; without it that wave runs unsplit.
size_t tc_apply_tail_bytes(int lp);
int launch_tc_apply(const float *A, int64_t m, int64_t n, int64_t lda, const __nv_bfloat16 *xsplit, int lp,
                    float *Y, DevStatus *st, cudaStream_t s, const float *bias = nullptr,
                    float *tail_part = nullptr);
// part[s] (n x lp) = A^T Q over the rows of split s, Q given pre-split.
int launch_tc_adjoint(const float *A, int64_t m, int64_t n, int64_t lda, const __nv_bfloat16 *qsplit, int lp,
                      float *part, int splits, DevStatus *st, cudaStream_t s);

// The renormalisations' tall-skinny products on the tensor cores, split in three
// BF16 pieces (exact) with the six products of order <= 2^-18: FP32 accuracy.
constexpr int64_t kTcRenormMinRows = 16384;            // shorter blocks stay on the SIMT kernels
bool tc_gram_ok(int64_t rows, int lp);                 // lp <= 128
bool tc_rmul_ok(int64_t rows, int ncols);              // ncols <= 256
size_t tc_rmul_split_bytes(int lp);
// part[s] (lp x lp) = Y^T Y over the rows of split s (*splits_out of them); nothing
// when skip && *skip == 0.
int launch_tc_gram(const float *Y, int64_t rows, int lp, float *part, int *splits_out, const int *skip,
                   DevStatus *st, cudaStream_t s);
// out (rows x ncols, leading dimension ldo) = Y R with Y rows x lp (leading dimension
// lp) and R lp x ncols (leading dimension ldr), ncols <= lp; R is split into rsplit
// (tc_rmul_split_bytes(lp) bytes).  With skip (square R, ncols == ldo == lp) the
// product is the identity when *skip == 0: out = Y, as launch_sgemm's copy flag.
int launch_tc_rmul(const float *Y, int64_t rows, int lp, const float *R, int64_t ldr, int ncols,
                   __nv_bfloat16 *rsplit, float *out, int64_t ldo, const int *skip, DevStatus *st, cudaStream_t s);

}  // namespace rpca

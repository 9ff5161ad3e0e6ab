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
// Y (m x lp) = A X, X given pre-split.
int launch_tc_apply(const float *A, int64_t m, int64_t n, int64_t lda, const __nv_bfloat16 *xsplit, int lp,
                    float *Y, DevStatus *st, cudaStream_t s);
// part[s] (n x lp) = A^T Q over the rows of split s, Q given pre-split.
int launch_tc_adjoint(const float *A, int64_t m, int64_t n, int64_t lda, const __nv_bfloat16 *qsplit, int lp,
                      float *part, int splits, DevStatus *st, cudaStream_t s);

}  // namespace rpca

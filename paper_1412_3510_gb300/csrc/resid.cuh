// Residual estimator (Section 4) shared by the dense and sparse entry points.
#pragma once

#include "pipeline.cuh"

namespace rpca {

struct ResidLayout {
    int64_t m = 0, n = 0;
    int k = 0, s_adj = 1, mchunks = 0, nchunks = 0;
    size_t status = 0, x8 = 0, z8 = 0, w8 = 0, q8 = 0, part = 0, wpart = 0, ypart = 0, tpart = 0,
           t2part = 0, npart = 0, total = 0;
};

ResidLayout make_resid_layout(int64_t m, int64_t n, int k, int adj_splits);

int run_resid(const Operator &op, int raw, const float *U, int64_t ldu, const float *S, const float *V,
              int64_t ldv, int k, int iters, uint64_t seed, double *est, void *ws, const ResidLayout &R,
              cudaStream_t s, bool clear_status = true);

}  // namespace rpca

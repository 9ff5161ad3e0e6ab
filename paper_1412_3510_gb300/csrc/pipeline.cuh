// The randomized PCA pipeline shared by the dense and sparse entry points.
#pragma once

#include "internal.cuh"

namespace rpca {

// The two products the method needs, for one storage format of A.
struct Operator {
    int64_t m = 0, n = 0;
    void *scratch = nullptr;          // operator-owned part of the workspace
    DevStatus *st = nullptr;          // device status block
    virtual ~Operator() = default;
    virtual size_t scratch_bytes(int lp) const { (void)lp; return 0; }
    // Y (m x lp) = A X (X n x lp); padding columns of X are zero.  bias (lp values,
    // only when fuses_bias()): Y = A X - 1 bias, the implicit centring.
    virtual int apply(const float *X, int lp, float *Y, cudaStream_t s, const float *bias = nullptr) const = 0;
    virtual bool fuses_bias() const { return false; }
    // True when the bias c X matches the product's own row mean to FP32 rounding (the
    // column means come from an FP32-accumulated adjoint product).  Otherwise the
    // block that becomes the final Q, whose ones-direction component reaches U
    // unfiltered, is centred on its own row mean instead.
    virtual bool exact_bias(int lp) const { (void)lp; return false; }
    // part / X: X (n x lp) = A^T Q as `splits` partial slices in `part`
    // (n x lp each), or written directly when splits() == 0.
    virtual int adjoint(const float *Q, int lp, float *part, cudaStream_t s) const = 0;
    virtual int adjoint_splits(int lp) const = 0;   // 0: adjoint writes X directly into part
};

struct Layout {
    int64_t m = 0, n = 0;
    int l = 0, lp = 0, k = 0, kp = 0;
    int s_adj = 0, s_gram_m = 0, s_gram_n = 0, cchunks = 0;
    size_t status = 0, x0 = 0, x1 = 0, y0 = 0, y1 = 0, part = 0, cpart = 0, qpart = 0, G = 0,
           rinv = 0, racc0 = 0, racc1 = 0, wk = 0, zk = 0, sig = 0, perm = 0, rot = 0, zbuf = 0,
           rinv_m = 0, flags = 0, scal = 0, cvec = 0, bias = 0, bpart = 0, r32 = 0, wfull = 0, zfull = 0, svd64 = 0, lu0 = 0,
           lu1 = 0, rsplit = 0, scratch = 0, total = 0;
};

Layout make_layout(int64_t m, int64_t n, int l, int k, int adjoint_splits, size_t op_scratch);

// Validate the arguments common to every entry point.
int check_common(int64_t m, int64_t n, const rpca_opts *o, const float *U, int64_t ldu,
                 const float *S, const float *V, int64_t ldv, const void *ws, size_t ws_bytes,
                 size_t need);

// Run the whole method (Sections 2 and 5; Eqs. i1-i4) on operator `op`.
int run_pipeline(Operator &op, const rpca_opts *o, float *U, int64_t ldu, float *S, float *V,
                 int64_t ldv, void *ws, const Layout &L, cudaStream_t s, bool clear_status = true);

// Self-adjoint A (m == n): Section 5's loop (products with A only), then either the
// two-sided projection B = Q^T A Q and its SVD (nystrom == false: A ~ U diag(S) V^T with
// V = U diag(sign(lambda))), or Section 3's stabilised Nystrom method (nystrom == true:
// A ~ U diag(S) U^T, V unused).
int run_pipeline_sym(Operator &op, const rpca_opts *o, bool nystrom, float *U, int64_t ldu, float *S, float *V,
                     int64_t ldv, void *ws, const Layout &L, cudaStream_t s);

// Renormalisation kind and the odd-only flag of rpca_opts::renorm.
inline int renorm_kind(int renorm) { return renorm & ~RPCA_RENORM_ODD_ONLY; }
inline bool renorm_odd_only(int renorm) { return (renorm & RPCA_RENORM_ODD_ONLY) != 0; }

// Offset of the small SVD's singular values in rpca_dense's workspace.
size_t dense_sigma_offset(int64_t m, int64_t n, const float *A, int64_t lda, const rpca_opts *o);

}  // namespace rpca

// Dense entry point: A is an m x n FP32 row-major matrix (leading dimension lda).
#include "pipeline.cuh"
#include "resid.cuh"
#include "tc_gemm.cuh"
#include "timing.cuh"

namespace rpca {

namespace {

// The two passes over A.  FP32: register-blocked FFMA kernels.  BF16X3: the
// tcgen05 split-BF16 kernels (the block operand is split once per pass into
// the operator's scratch); A must then be 16-byte aligned with lda % 4 == 0.
struct DenseOp final : Operator {
    const float *A = nullptr;
    int64_t lda = 0;
    int precision = RPCA_PREC_FP32;

    bool tc(int lp) const { return precision == RPCA_PREC_BF16X3 && tc_supported(A, lda, lp); }
    size_t scratch_bytes(int lp) const override {
        if (precision != RPCA_PREC_BF16X3) return 0;
        return std::max(apply_tail_offset(lp) + tc_apply_tail_bytes(lp), tc_split_bytes(m, lp));
    }
    // A X's scratch: the split X, then the K pieces of the last wave's row tiles
    size_t apply_tail_offset(int lp) const { return (tc_split_bytes(n, lp) + 255) & ~(size_t)255; }
    int apply(const float *X, int lp, float *Y, cudaStream_t s, const float *bias) const override {
        if (tc(lp)) {
            auto *xs = reinterpret_cast<__nv_bfloat16 *>(scratch);
            RPCA_TRY(launch_tc_split(X, n, lp, xs, s));
            TimedScope ts(kTimeApplyKernel, s);
            float *tail = reinterpret_cast<float *>(reinterpret_cast<char *>(scratch) + apply_tail_offset(lp));
            return launch_tc_apply(A, m, n, lda, xs, lp, Y, st, s, bias, tail);
        }
        TimedScope ts(kTimeApplyKernel, s);
        return launch_sgemm(false, m, lp, n, A, lda, X, lp, Y, lp, 1, 0, s, nullptr, bias);
    }
    bool fuses_bias() const override { return true; }
    // the tensor cores' FP32 accumulation drifts (about 2^-27 per K element, chunked at
    // 2048), which puts up to ~1e-5 relative error into the column means c = A^T 1 / m
    bool exact_bias(int lp) const override { return !tc(lp); }
    int adjoint_splits(int lp) const override {
        return tc(lp) ? tc_adjoint_splits(n, m, lp) : choose_splits(n, lp, m);
    }
    int adjoint(const float *Q, int lp, float *part, cudaStream_t s) const override {
        const int sp = adjoint_splits(lp);
        if (tc(lp)) {
            auto *qs = reinterpret_cast<__nv_bfloat16 *>(scratch);
            RPCA_TRY(launch_tc_split(Q, m, lp, qs, s));
            TimedScope ts(kTimeAdjointKernel, s);
            return launch_tc_adjoint(A, m, n, lda, qs, lp, part, sp, st, s);
        }
        TimedScope ts(kTimeAdjointKernel, s);
        return launch_sgemm(true, n, lp, m, A, lda, Q, lp, part, lp, sp, n * (int64_t)lp, s);
    }
};

}  // namespace

}  // namespace rpca

extern "C" size_t rpca_dense_workspace_size(int64_t m, int64_t n, const rpca_opts *o) {
    if (!o || m < 1 || n < 1 || o->l < 1 || o->k < 1 || o->l > RPCA_MAX_L) return 0;
    const int lp = rpca::padded_l(o->l);
    // sized for the larger of the two forms' partial buffers so that the
    // same workspace serves either precision
    const int splits = std::max(rpca::choose_splits(n, lp, m), rpca::tc_adjoint_splits(n, m, lp));
    rpca::DenseOp op;
    op.m = m; op.n = n; op.precision = rpca::pass_precision(o->precision);
    return rpca::make_layout(m, n, o->l, o->k, splits, op.scratch_bytes(lp)).total;
}

extern "C" int rpca_dense(const float *A, int64_t m, int64_t n, int64_t lda, const rpca_opts *o,
                          float *U, int64_t ldu, float *S, float *V, int64_t ldv, void *ws,
                          size_t ws_bytes, rpca_stream_t stream) {
    if (!A || !o || lda < n) return RPCA_ERR_INVALID_ARG;
    const size_t need = rpca_dense_workspace_size(m, n, o);
    RPCA_TRY(rpca::check_common(m, n, o, U, ldu, S, V, ldv, ws, ws_bytes, need));
    if (rpca::renorm_kind(o->renorm) == RPCA_RENORM_LU && !rpca::tslu_supported(o->l)) return RPCA_ERR_UNSUPPORTED;
    rpca::DenseOp op;
    op.m = m; op.n = n; op.A = A; op.lda = lda; op.precision = rpca::pass_precision(o->precision);
    const int lp = rpca::padded_l(o->l);
    const int splits = std::max(rpca::choose_splits(n, lp, m), rpca::tc_adjoint_splits(n, m, lp));
    const rpca::Layout L = rpca::make_layout(m, n, o->l, o->k, splits, op.scratch_bytes(lp));
    return rpca::run_pipeline(op, o, U, ldu, S, V, ldv, ws, L, (cudaStream_t)stream);
}

namespace {

// The arguments of rpca_sym and rpca_nystrom: a square A used as it is.
int check_sym(const float *A, int64_t n, int64_t lda, const rpca_opts *o, const float *U, int64_t ldu,
              const float *S, const void *ws, size_t ws_bytes) {
    if (!A || !o || !U || !S || n < 1 || lda < n) return RPCA_ERR_INVALID_ARG;
    if (!o->raw || o->its < 1) return RPCA_ERR_INVALID_ARG;
    const size_t need = rpca_sym_workspace_size(n, o);
    // check_common validates k, l, its, precision and renorm; V is checked by the caller
    return rpca::check_common(n, n, o, U, ldu, S, U, ldu, ws, ws_bytes, need);
}

int run_sym(const float *A, int64_t n, int64_t lda, const rpca_opts *o, bool nystrom, float *U, int64_t ldu,
            float *S, float *V, int64_t ldv, void *ws, rpca_stream_t stream) {
    if (rpca::renorm_kind(o->renorm) == RPCA_RENORM_LU && !rpca::tslu_supported(o->l)) return RPCA_ERR_UNSUPPORTED;
    rpca::DenseOp op;
    op.m = n; op.n = n; op.A = A; op.lda = lda; op.precision = rpca::pass_precision(o->precision);
    const int lp = rpca::padded_l(o->l);
    const int splits = std::max(rpca::choose_splits(n, lp, n), rpca::tc_adjoint_splits(n, n, lp));
    const rpca::Layout L = rpca::make_layout(n, n, o->l, o->k, splits, op.scratch_bytes(lp));
    return rpca::run_pipeline_sym(op, o, nystrom, U, ldu, S, V, ldv, ws, L, (cudaStream_t)stream);
}

}  // namespace

extern "C" size_t rpca_sym_workspace_size(int64_t n, const rpca_opts *o) { return rpca_dense_workspace_size(n, n, o); }

extern "C" int rpca_sym(const float *A, int64_t n, int64_t lda, const rpca_opts *o, float *U, int64_t ldu,
                        float *S, float *V, int64_t ldv, void *ws, size_t ws_bytes, rpca_stream_t stream) {
    RPCA_TRY(check_sym(A, n, lda, o, U, ldu, S, ws, ws_bytes));
    if (!V || ldv < o->k) return RPCA_ERR_INVALID_ARG;
    return run_sym(A, n, lda, o, false, U, ldu, S, V, ldv, ws, stream);
}

extern "C" int rpca_nystrom(const float *A, int64_t n, int64_t lda, const rpca_opts *o, float *U, int64_t ldu,
                            float *S, void *ws, size_t ws_bytes, rpca_stream_t stream) {
    RPCA_TRY(check_sym(A, n, lda, o, U, ldu, S, ws, ws_bytes));
    return run_sym(A, n, lda, o, true, U, ldu, S, nullptr, 0, ws, stream);
}

namespace rpca {

// Byte offset, within rpca_dense's workspace, of the l singular values of the
// small SVD (descending), valid after rpca_dense has run with the same arguments.
size_t dense_sigma_offset(int64_t m, int64_t n, const float *A, int64_t lda, const rpca_opts *o) {
    DenseOp op;
    op.m = m; op.n = n; op.A = A; op.lda = lda; op.precision = rpca::pass_precision(o->precision);
    const int lp = padded_l(o->l);
    const int splits = std::max(choose_splits(n, lp, m), tc_adjoint_splits(n, m, lp));
    return make_layout(m, n, o->l, o->k, splits, op.scratch_bytes(lp)).sig;
}

}  // namespace rpca

extern "C" size_t rpca_resid_workspace_size(int64_t m, int64_t n, int32_t k) {
    if (m < 1 || n < 1 || k < 0 || k > RPCA_MAX_L) return 0;
    return rpca::make_resid_layout(m, n, k, rpca::choose_splits(n, 8, m)).total;
}

extern "C" int rpca_resid_norm(const float *A, int64_t m, int64_t n, int64_t lda, int32_t raw,
                               const float *U, int64_t ldu, const float *S, const float *V, int64_t ldv,
                               int32_t k, int32_t iters, uint64_t seed, double *est, void *ws,
                               size_t ws_bytes, rpca_stream_t stream) {
    if (!A || !est || m < 1 || n < 1 || lda < n || k < 0 || k > RPCA_MAX_L || iters < 1) return RPCA_ERR_INVALID_ARG;
    if (k > 0 && (!U || !S || !V || ldu < k || ldv < k)) return RPCA_ERR_INVALID_ARG;
    const size_t need = rpca_resid_workspace_size(m, n, k);
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0 || ws_bytes < need) return RPCA_ERR_WORKSPACE;
    rpca::DenseOp op;
    op.m = m; op.n = n; op.A = A; op.lda = lda;
    const rpca::ResidLayout R = rpca::make_resid_layout(m, n, k, op.adjoint_splits(8));
    return rpca::run_resid(op, raw, U, ldu, S, V, ldv, k, iters, seed, est, ws, R, (cudaStream_t)stream);
}

namespace {

struct PassPlan {
    size_t status = 0, part = 0, scratch = 0, total = 0;
    int splits = 1;
};

PassPlan pass_plan(const rpca::DenseOp &op, int w, int adjoint) {
    PassPlan P;
    auto a256 = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t off = 0;
    P.status = off; off = a256(off + sizeof(rpca::DevStatus));
    P.splits = adjoint ? std::max(op.adjoint_splits(w), 1) : 1;
    // room for either form's number of partial slices
    const int most = std::max(rpca::choose_splits(op.n, w, op.m), rpca::tc_adjoint_splits(op.n, op.m, w));
    P.part = off; off = a256(off + (adjoint ? (size_t)most * op.n * w * 4 : 0));
    P.scratch = off; off = a256(off + op.scratch_bytes(w));
    P.total = off;
    return P;
}

}  // namespace

extern "C" size_t rpca_dense_pass_workspace_size(int64_t m, int64_t n, int32_t w, int32_t adjoint,
                                                 int32_t precision) {
    if (m < 1 || n < 1 || w < 8 || w > 256 || w % 8) return 0;
    rpca::DenseOp op;
    op.m = m; op.n = n; op.precision = precision;
    op.A = reinterpret_cast<const float *>(256); op.lda = 4;       // size as if the tensor-core form runs
    return pass_plan(op, w, adjoint).total;
}

extern "C" int rpca_dense_pass(const float *A, int64_t m, int64_t n, int64_t lda, int32_t adjoint, const float *B,
                               int32_t w, float *C, int32_t precision, void *ws, size_t ws_bytes,
                               rpca_stream_t stream) {
    if (!A || !B || !C || m < 1 || n < 1 || lda < n || w < 8 || w > 256 || w % 8) return RPCA_ERR_INVALID_ARG;
    if (precision != RPCA_PREC_FP32 && precision != RPCA_PREC_BF16X3) return RPCA_ERR_INVALID_ARG;
    const size_t need = rpca_dense_pass_workspace_size(m, n, w, adjoint, precision);
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0 || ws_bytes < need) return RPCA_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    rpca::DenseOp op;
    op.m = m; op.n = n; op.A = A; op.lda = lda; op.precision = precision;
    const PassPlan P = pass_plan(op, w, adjoint);
    char *base = reinterpret_cast<char *>(ws);
    op.st = reinterpret_cast<rpca::DevStatus *>(base + P.status);
    op.scratch = base + P.scratch;
    if (cudaMemsetAsync(op.st, 0, sizeof(rpca::DevStatus), s) != cudaSuccess) return RPCA_ERR_CUDA;
    if (!adjoint) return op.apply(B, w, C, s, nullptr);
    float *part = reinterpret_cast<float *>(base + P.part);
    RPCA_TRY(op.adjoint(B, w, part, s));
    return rpca::launch_adjoint_reduce(part, P.splits, n, w, w, C, 0, (double)m, nullptr, 0, s);
}

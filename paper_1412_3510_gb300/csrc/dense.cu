// Dense entry point: A is an m x n FP32 row-major matrix (leading dimension lda).
#include "pipeline.cuh"

namespace rpca {

namespace {

struct DenseOp final : Operator {
    const float *A = nullptr;
    int64_t lda = 0;
    int precision = RPCA_PREC_FP32;

    int apply(const float *X, int lp, float *Y, cudaStream_t s) const override {
        return launch_sgemm(false, m, lp, n, A, lda, X, lp, Y, lp, 1, 0, s);
    }
    int adjoint_splits(int lp) const override { return choose_splits(n, lp, m); }
    int adjoint(const float *Q, int lp, float *part, cudaStream_t s) const override {
        const int sp = adjoint_splits(lp);
        return launch_sgemm(true, n, lp, m, A, lda, Q, lp, part, lp, sp, n * (int64_t)lp, s);
    }
};

}  // namespace

}  // namespace rpca

extern "C" size_t rpca_dense_workspace_size(int64_t m, int64_t n, const rpca_opts *o) {
    if (!o || m < 1 || n < 1 || o->l < 1 || o->k < 1 || o->l > RPCA_MAX_L) return 0;
    const int lp = rpca::padded_l(o->l);
    return rpca::make_layout(m, n, o->l, o->k, rpca::choose_splits(n, lp, m)).total;
}

extern "C" int rpca_dense(const float *A, int64_t m, int64_t n, int64_t lda, const rpca_opts *o,
                          float *U, int64_t ldu, float *S, float *V, int64_t ldv, void *ws,
                          size_t ws_bytes, rpca_stream_t stream) {
    if (!A || !o || lda < n) return RPCA_ERR_INVALID_ARG;
    const size_t need = rpca_dense_workspace_size(m, n, o);
    RPCA_TRY(rpca::check_common(m, n, o, U, ldu, S, V, ldv, ws, ws_bytes, need));
    if (o->precision != RPCA_PREC_FP32 || o->renorm != RPCA_RENORM_CHOLQR) return RPCA_ERR_UNSUPPORTED;
    rpca::DenseOp op;
    op.m = m; op.n = n; op.A = A; op.lda = lda; op.precision = o->precision;
    const int lp = rpca::padded_l(o->l);
    const rpca::Layout L = rpca::make_layout(m, n, o->l, o->k, op.adjoint_splits(lp));
    return rpca::run_pipeline(op, o, U, ldu, S, V, ldv, ws, L, (cudaStream_t)stream);
}

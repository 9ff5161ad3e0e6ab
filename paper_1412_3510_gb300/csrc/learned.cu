// Dense randomized PCA with the learned sketch weighting and its fallback.
//
// features -> MLP -> d; the method of Sections 2 and 5 with diag(d) Omega;
// the power-method residual estimate of Section 4; if the estimate is above
// fallback_ratio * s_{k+1} (s_{k+1}: the (k+1)-th singular value of the rank-l
// approximation, the best the rank-k output could do on the sketched range)
// the plain Gaussian sketch runs instead.
//
// Workspace: [MLP status | s_{k+1} | estimate | d (n) | F (n x 16) | shared rest], the rest
// reused in turn by the features pass, rpca_dense and the estimator.
#include "internal.cuh"
#include "pipeline.cuh"

namespace rpca {
namespace {

struct LearnedPlan {
    size_t mlp_status = 0, sk1 = 0, est = 0, d = 0, F = 0, rest = 0, rest_bytes = 0, total = 0;
};

LearnedPlan learned_plan(int64_t m, int64_t n, const rpca_opts *o) {
    LearnedPlan P;
    auto a256 = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t off = 0;
    P.mlp_status = off; off = a256(off + rpca_mlp_forward_workspace_size());
    P.sk1 = off; off = a256(off + sizeof(float));
    P.est = off; off = a256(off + sizeof(double));
    P.d = off; off = a256(off + (size_t)n * sizeof(float));
    P.F = off; off = a256(off + (size_t)n * RPCA_MLP_FEATURES * sizeof(float));
    P.rest = off;
    P.rest_bytes = std::max({rpca_features_workspace_size(m, n), rpca_dense_workspace_size(m, n, o),
                             rpca_resid_workspace_size(m, n, o->k)});
    P.total = off + P.rest_bytes;
    return P;
}

}  // namespace
}  // namespace rpca

using namespace rpca;

extern "C" size_t rpca_dense_learned_workspace_size(int64_t m, int64_t n, const rpca_opts *o) {
    if (!o || m < 1 || n < 1 || rpca_dense_workspace_size(m, n, o) == 0) return 0;
    return learned_plan(m, n, o).total;
}

extern "C" int rpca_dense_learned(const float *A, int64_t m, int64_t n, int64_t lda, const rpca_opts *o,
                                  const void *mlp_packed, int32_t resid_iters, double fallback_ratio, float *U,
                                  int64_t ldu, float *S, float *V, int64_t ldv, double *est_out, void *ws,
                                  size_t ws_bytes, rpca_stream_t stream) {
    if (!A || !o || !mlp_packed || (reinterpret_cast<uintptr_t>(mlp_packed) & 15u) || lda < n || m < 1 || n < 1 ||
        resid_iters < 1 || !(fallback_ratio > 0.0) || o->omega || o->col_weights)
        return RPCA_ERR_INVALID_ARG;
    const size_t need = rpca_dense_learned_workspace_size(m, n, o);
    if (need == 0) return RPCA_ERR_INVALID_ARG;
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0 || ws_bytes < need) return RPCA_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    const LearnedPlan P = learned_plan(m, n, o);
    char *base = static_cast<char *>(ws);
    char *rest = base + P.rest;
    float *d = reinterpret_cast<float *>(base + P.d);
    float *F = reinterpret_cast<float *>(base + P.F);
    float *sk1 = reinterpret_cast<float *>(base + P.sk1);
    double *est_dev = reinterpret_cast<double *>(base + P.est);

    RPCA_TRY(rpca_sketch_features(A, m, n, lda, o->raw, o->seed, F, rest, P.rest_bytes, stream));
    RPCA_TRY(rpca_mlp_forward(mlp_packed, F, n, nullptr, d, base + P.mlp_status,
                              rpca_mlp_forward_workspace_size(), stream));
    rpca_opts ol = *o;
    ol.col_weights = d;
    int rc = rpca_dense(A, m, n, lda, &ol, U, ldu, S, V, ldv, rest, P.rest_bytes, stream);
    if (rc < 0) return rc;
    const bool check = o->l > o->k;
    if (check) {
        const size_t off = dense_sigma_offset(m, n, A, lda, &ol) + (size_t)o->k * sizeof(float);
        if (cudaMemcpyAsync(sk1, rest + off, sizeof(float), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return RPCA_ERR_CUDA;
    }
    // the dense run's device status (shifted CholeskyQR, Jacobi sweeps, ...) before the
    // estimator reuses the workspace
    int32_t dense_status = 0;
    RPCA_TRY(rpca_read_status(rest, stream, &dense_status));
    if (dense_status < 0) return dense_status;
    int32_t mlp_status = 0;
    RPCA_TRY(rpca_read_status(base + P.mlp_status, stream, &mlp_status));
    if (mlp_status < 0) return mlp_status;

    RPCA_TRY(rpca_resid_norm(A, m, n, lda, o->raw, U, ldu, S, V, ldv, o->k, resid_iters, o->seed, est_dev, rest,
                             P.rest_bytes, stream));
    double est = 0.0;
    float sk1_host = 0.f;
    if (cudaMemcpyAsync(&est, est_dev, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        (check && cudaMemcpyAsync(&sk1_host, sk1, sizeof(float), cudaMemcpyDeviceToHost, s) != cudaSuccess) ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return RPCA_ERR_CUDA;
    int32_t resid_status = 0;
    RPCA_TRY(rpca_read_status(rest, stream, &resid_status));
    if (resid_status < 0) return resid_status;
    if (est_out) {
        est_out[0] = est;
        est_out[1] = (double)sk1_host;
    }
    if (check && est > fallback_ratio * (double)sk1_host) {
        rc = rpca_dense(A, m, n, lda, o, U, ldu, S, V, ldv, rest, P.rest_bytes, stream);
        return rc < 0 ? rc : RPCA_FELL_BACK;
    }
    return RPCA_OK;
}

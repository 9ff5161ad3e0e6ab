// The randomized PCA of Szlam, Kluger & Tygert (2014), Sections 2 and 5, as a
// sequence of launches on one stream:
//
//   Omega (Philox)                      Section 2 test vectors
//   Y = A_c Omega                       the sketch
//   Q = renorm(Y)                       Section 5: renormalise every product
//   its times: X = A_c^* Q; Q' = renorm(X); Y = A_c Q'; Q = renorm(Y)
//   the last renormalisation is a full orthonormalisation (Section 5's QR),
//   here CholeskyQR applied two times, three when the first had to shift
//
// A renormalisation Q = Y R^-1 on the m side that only feeds the next
// adjoint product is never formed: A_c^* (Y R^-1) = (A_c^* Y) R^-1, so R^-1
// is applied to the small n x l result instead.
//   B^* = A_c^* Q; B^* = Q2 R (CholeskyQR x3); R^T = W Sigma Z^T (Jacobi)
//   V = Q2 Z, U = Q W (Eq. i4), first k columns, sign convention on V.
//
// Blocks on the m side (Y, Q) and the n side (X, Q') are FP32, row-major with
// the padded width lp = round_up(l + 1, 8); column l of a Q that enters an
// adjoint product holds ones (it carries m c through A^T), every other padding
// column holds zeros.
#include "pipeline.cuh"
#include "tc_gemm.cuh"
#include "timing.cuh"

namespace rpca {

namespace {

__global__ void copy_scale_kernel(int64_t n, int l, const float *__restrict__ src, int64_t lds,
                                  const float *__restrict__ w, float *__restrict__ dst, int64_t ldd) {
    const int64_t total = n * (int64_t)l;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / l;
        const int j = (int)(e % l);
        float v = src[i * lds + j];
        if (w) v *= w[i];
        dst[i * ldd + j] = v;
    }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

Layout make_layout(int64_t m, int64_t n, int l, int k, int adjoint_splits, size_t op_scratch) {
    Layout L;
    L.m = m; L.n = n; L.l = l; L.k = k;
    L.lp = padded_l(l);
    L.kp = (int)round_up(k, 4);
    L.s_adj = adjoint_splits;
    L.s_gram_m = gram_splits(m, L.lp);
    L.s_gram_n = gram_splits(n, L.lp);
    L.cchunks = colsum_chunks(m);
    const size_t lp = (size_t)L.lp;
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t o = off; off = align256(off + bytes); return o; };
    L.status = take(sizeof(DevStatus));
    L.x0 = take((size_t)n * lp * 4);
    L.x1 = take((size_t)n * lp * 4);
    L.y0 = take((size_t)m * lp * 4);
    L.y1 = take((size_t)m * lp * 4);
    size_t part = std::max({(size_t)std::max(L.s_adj, 1) * (size_t)n * lp,
                            (size_t)L.s_gram_m * lp * lp, (size_t)L.s_gram_n * lp * lp});
    L.part = take(part * 4);
    L.cpart = take((size_t)L.cchunks * l * 4);
    L.qpart = take((size_t)L.cchunks * l * 4);
    L.G = take((size_t)gram_ld(l) * gram_ld(l) * 4);
    L.rinv = take(lp * lp * 4);
    L.racc0 = take((size_t)l * l * 4);
    L.racc1 = take((size_t)l * l * 4);
    L.wk = take(lp * L.kp * 4);
    L.zk = take(lp * L.kp * 4);
    L.sig = take(lp * 4);
    L.perm = take(lp * 4);
    L.rot = take(small_svd_rot_floats(l) * 4);
    L.zbuf = take(256);
    L.rinv_m = take(lp * lp * 4);
    L.flags = take(256);
    L.lu0 = take(tslu_ids_bytes(std::max(m, n), l));
    L.lu1 = take(tslu_ids_bytes(std::max(m, n), l));
    L.rsplit = take(tc_rmul_split_bytes(L.lp));
    L.scratch = take(op_scratch);
    L.total = off;
    return L;
}

int check_common(int64_t m, int64_t n, const rpca_opts *o, const float *U, int64_t ldu,
                 const float *S, const float *V, int64_t ldv, const void *ws, size_t ws_bytes,
                 size_t need) {
    if (!o || !U || !S || !V) return RPCA_ERR_INVALID_ARG;
    if (m < 1 || n < 1) return RPCA_ERR_INVALID_ARG;
    if (o->k < 1 || o->l < o->k || o->l > RPCA_MAX_L || (int64_t)o->l > std::min(m, n)) return RPCA_ERR_INVALID_ARG;
    if (o->its < 0 || o->its > 1000) return RPCA_ERR_INVALID_ARG;
    if (ldu < o->k || ldv < o->k) return RPCA_ERR_INVALID_ARG;
    if (o->precision != RPCA_PREC_FP32 && o->precision != RPCA_PREC_BF16X3) return RPCA_ERR_INVALID_ARG;
    if (o->renorm != RPCA_RENORM_CHOLQR && o->renorm != RPCA_RENORM_LU) return RPCA_ERR_INVALID_ARG;
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0 || ws_bytes < need) return RPCA_ERR_WORKSPACE;
    return RPCA_OK;
}

namespace {

struct Ctx {
    const Layout &L;
    char *ws;
    cudaStream_t s;
    DevStatus *st;
    bool lu = false;          // non-final renormalisations by tall-skinny LU
    template <class T> T *at(size_t off) const { return reinterpret_cast<T *>(ws + off); }
};

// Gram, reduction and Cholesky of a tall block: rinv = R^-1 with in^T in = R^T R.
int gram_chol(const Ctx &c, const float *in, int64_t rows, int splits, float *rinv, const float *racc_in,
              float *racc_out, int *shifted_out, const int *skip) {
    const Layout &L = c.L;
    const int lp = L.lp;
    float *part = c.at<float>(L.part);
    float *G = c.at<float>(L.G);
    {
        TimedScope ts(kTimeGram, c.s);
        if (tc_gram_ok(rows, lp)) {
            RPCA_TRY(launch_tc_gram(in, rows, lp, part, &splits, skip, c.st, c.s));
        } else {
            RPCA_TRY(launch_gram(in, rows, lp, part, splits, skip, c.s));
        }
        RPCA_TRY(launch_gram_reduce(part, splits, L.l, lp, G, c.s, skip));
    }
    TimedScope ts(kTimeChol, c.s);
    return launch_chol_inv(G, L.l, lp, rinv, racc_in, racc_out, c.st, c.s, shifted_out, skip);
}

// Tall-skinny LU of a block: rinv = U^-1 with in = P^T L U (tournament pivoting).
int lu_factor(const Ctx &c, const float *in, int64_t rows, float *rinv) {
    const Layout &L = c.L;
    TimedScope ts(kTimeChol, c.s);
    const int32_t *winner = nullptr;
    RPCA_TRY(launch_tslu_select(in, rows, L.lp, L.l, c.at<int32_t>(L.lu0), c.at<int32_t>(L.lu1), &winner, c.s));
    return launch_lu_final(in, rows, L.lp, L.l, winner, rinv, c.st, c.s);
}

// One CholeskyQR round: out = in R^-1.  With skip (*skip == 0 on the device) the round is
// the identity and out = in.
int cholqr_round(const Ctx &c, const float *in, float *out, int64_t rows, int splits, const float *racc_in,
                 float *racc_out, int *shifted_out = nullptr, const int *skip = nullptr) {
    const Layout &L = c.L;
    const int lp = L.lp;
    float *rinv = c.at<float>(L.rinv);
    RPCA_TRY(gram_chol(c, in, rows, splits, rinv, racc_in, racc_out, shifted_out, skip));
    TimedScope ts(kTimeTrsm, c.s);
    if (tc_rmul_ok(rows, lp))
        return launch_tc_rmul(in, rows, lp, rinv, lp, lp, c.at<__nv_bfloat16>(L.rsplit), out, lp, skip, c.st, c.s);
    RPCA_TRY(launch_sgemm(false, rows, lp, lp, in, lp, rinv, lp, out, lp, 1, 0, c.s, skip));
    return RPCA_OK;
}

// m-side renormalisation of y0 (a fresh product A X).  Non-final: y0 is centred
// and kept, R^-1 goes to rinv_m for the next adjoint product (implicit Q).
// Final: explicit orthonormal Q in y1 (CholeskyQR two or three times).
// Returns through *q the block the next adjoint product reads.
int renorm_m(const Ctx &c, bool raw, bool final_, const float **q, bool *pending) {
    const Layout &L = c.L;
    float *y0 = c.at<float>(L.y0), *y1 = c.at<float>(L.y1);
    int *flag = c.at<int>(L.flags);
    if (!raw) {
        TimedScope ts(kTimeCentre, c.s);
        int nch = 0;
        RPCA_TRY(launch_colsum_partial(y0, L.m, L.l, L.lp, c.at<float>(L.cpart), &nch, c.s));
        RPCA_TRY(launch_center(y0, L.m, L.l, L.lp, c.at<float>(L.cpart), nch, c.s));
    }
    float *qout = y1;
    if (!final_) {
        if (c.lu) RPCA_TRY(lu_factor(c, y0, L.m, c.at<float>(L.rinv_m)));
        else RPCA_TRY(gram_chol(c, y0, L.m, L.s_gram_m, c.at<float>(L.rinv_m), nullptr, nullptr, nullptr, nullptr));
        qout = y0;
        *pending = true;
    } else {
        RPCA_TRY(cholqr_round(c, y0, y1, L.m, L.s_gram_m, nullptr, nullptr, flag));
        RPCA_TRY(cholqr_round(c, y1, y0, L.m, L.s_gram_m, nullptr, nullptr));
        RPCA_TRY(cholqr_round(c, y0, y1, L.m, L.s_gram_m, nullptr, nullptr, nullptr, flag));
        *pending = false;
    }
    RPCA_TRY(launch_finalize(qout, L.m, L.l, L.lp, raw ? 0.f : 1.f, raw ? nullptr : c.at<float>(L.qpart), c.s));
    *q = qout;
    return RPCA_OK;
}

// n-side renormalisation of x0 (a fresh product A^T Q) into x1; the final one
// accumulates the triangular factor R = R3 R2 R1 into racc0 (R3 = I when the
// first round did not shift).
int renorm_n(const Ctx &c, bool final_) {
    const Layout &L = c.L;
    float *x0 = c.at<float>(L.x0), *x1 = c.at<float>(L.x1);
    float *r0 = c.at<float>(L.racc0), *r1 = c.at<float>(L.racc1);
    int *flag = c.at<int>(L.flags) + 1;
    if (!final_ && c.lu) {
        float *rinv = c.at<float>(L.rinv);
        RPCA_TRY(lu_factor(c, x0, L.n, rinv));
        TimedScope ts(kTimeTrsm, c.s);
        return launch_sgemm(false, L.n, L.lp, L.lp, x0, L.lp, rinv, L.lp, x1, L.lp, 1, 0, c.s);
    }
    if (!final_) return cholqr_round(c, x0, x1, L.n, L.s_gram_n, nullptr, nullptr);
    RPCA_TRY(cholqr_round(c, x0, x1, L.n, L.s_gram_n, nullptr, r0, flag));
    RPCA_TRY(cholqr_round(c, x1, x0, L.n, L.s_gram_n, r0, r1));
    RPCA_TRY(cholqr_round(c, x0, x1, L.n, L.s_gram_n, r1, r0, nullptr, flag));
    return RPCA_OK;
}

// x0 = A_c^* q  (Section 5: (Q'*A)' - c'*(ones(1,m)*Q)), times the pending R^-1 of an
// implicit m-side renormalisation.
int adjoint_pass(const Operator &op, const Ctx &c, bool raw, const float *q, bool pending) {
    const Layout &L = c.L;
    float *part = c.at<float>(L.part);
    {
        TimedScope ts(kTimeAdjoint, c.s);
        RPCA_TRY(op.adjoint(q, L.lp, part, c.s));
    }
    const int splits = op.adjoint_splits(L.lp);
    float *dst = pending ? c.at<float>(L.x1) : c.at<float>(L.x0);
    RPCA_TRY(launch_adjoint_reduce(part, std::max(splits, 1), L.n, L.l, L.lp, dst, raw ? 0 : 1, (double)L.m,
                                   c.at<float>(L.qpart), L.cchunks, c.s));
    if (pending) {
        TimedScope ts(kTimeTrsm, c.s);
        RPCA_TRY(launch_sgemm(false, L.n, L.lp, L.lp, dst, L.lp, c.at<float>(L.rinv_m), L.lp, c.at<float>(L.x0), L.lp,
                              1, 0, c.s));
    }
    return RPCA_OK;
}

}  // namespace

int run_pipeline(Operator &op, const rpca_opts *o, float *U, int64_t ldu, float *S, float *V,
                 int64_t ldv, void *ws, const Layout &L, cudaStream_t s, bool clear_status) {
    Ctx c{L, reinterpret_cast<char *>(ws), s, reinterpret_cast<DevStatus *>(reinterpret_cast<char *>(ws) + L.status),
          o->renorm == RPCA_RENORM_LU};
    op.scratch = reinterpret_cast<char *>(ws) + L.scratch;
    op.st = c.st;
    const bool raw = o->raw != 0;
    const int l = L.l, lp = L.lp;
    float *x1 = c.at<float>(L.x1), *y0 = c.at<float>(L.y0), *y1 = c.at<float>(L.y1);

    if (clear_status && cudaMemsetAsync(c.st, 0, sizeof(DevStatus), s) != cudaSuccess) return RPCA_ERR_CUDA;
    if (cudaMemsetAsync(x1, 0, (size_t)L.n * lp * 4, s) != cudaSuccess) return RPCA_ERR_CUDA;

    // test matrix (Section 2), optionally weighted by d (Omega' = diag(d) Omega)
    if (o->omega) {
        const int64_t grid = std::min<int64_t>(cdiv(L.n * (int64_t)l, 256), (int64_t)num_sms() * 8);
        copy_scale_kernel<<<(unsigned)grid, 256, 0, s>>>(L.n, l, o->omega, l, o->col_weights, x1, lp);
        RPCA_CHECK_LAUNCH();
    } else {
        RPCA_TRY(launch_omega(L.n, l, o->seed, 0, o->col_weights, x1, lp, s));
    }

    auto apply = [&]() {
        TimedScope ts(kTimeApply, s);
        return op.apply(x1, lp, y0, s);
    };
    // sketch and power iterations
    const float *q = nullptr;
    bool pending = false;
    RPCA_TRY(apply());
    RPCA_TRY(renorm_m(c, raw, o->its == 0, &q, &pending));
    for (int it = 1; it <= o->its; ++it) {
        RPCA_TRY(adjoint_pass(op, c, raw, q, pending));
        RPCA_TRY(renorm_n(c, false));
        RPCA_TRY(apply());
        RPCA_TRY(renorm_m(c, raw, it == o->its, &q, &pending));
    }

    // B^* = A_c^* Q (Eq. i2), B^* = Q2 R, SVD of R^T (Eq. i3)
    RPCA_TRY(adjoint_pass(op, c, raw, q, pending));
    RPCA_TRY(renorm_n(c, true));
    float *wk = c.at<float>(L.wk), *zk = c.at<float>(L.zk), *sig = c.at<float>(L.sig);
    {
        TimedScope ts(kTimeSmallSvd, s);
        RPCA_TRY(launch_small_svd(c.at<float>(L.racc0), l, lp, L.k, L.kp, wk, zk, sig, c.at<float>(L.rot),
                                  c.at<float>(L.zbuf), c.at<int>(L.perm), c.st, s));
    }

    // V = Q2 Z_k, signs, U = Q W_k (Eq. i4)
    TimedScope ts_lift(kTimeLift, s);
    RPCA_TRY(launch_sgemm(false, L.n, L.k, lp, x1, lp, zk, L.kp, V, ldv, 1, 0, s));
    RPCA_TRY(launch_sign_fix(V, L.n, ldv, L.k, wk, lp, L.kp, sig, S, s));
    if (tc_rmul_ok(L.m, L.k) && (reinterpret_cast<uintptr_t>(U) & 3u) == 0)
        return launch_tc_rmul(y1, L.m, lp, wk, L.kp, L.k, c.at<__nv_bfloat16>(L.rsplit), U, ldu, nullptr, c.st, s);
    RPCA_TRY(launch_sgemm(false, L.m, L.k, lp, y1, lp, wk, L.kp, U, ldu, 1, 0, s));
    return RPCA_OK;
}

}  // namespace rpca

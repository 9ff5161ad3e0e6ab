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
#include <cmath>

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

// Symmetric part of the reduced l x l matrix G (row stride ldg): out[i][j] =
// (G[i][j] + G[j][i]) / 2 for i, j < l, row stride ldo, zero padding up to ldo.  With
// nu_out, also nu = nu_scale * trace(G) added to the diagonal and stored to *nu_out
// (the identity shift of the Nystrom method).  One CTA.
__global__ void __launch_bounds__(256)
symmetrize_kernel(const float *__restrict__ G, int l, int ldg, float *__restrict__ out, int ldo, float nu_scale,
                  float *__restrict__ nu_out, double *__restrict__ out64 = nullptr) {
    __shared__ float red[256];
    float nu = 0.f;
    if (nu_out) {
        float t = 0.f;
        for (int i = threadIdx.x; i < l; i += blockDim.x) t += G[(size_t)i * ldg + i];
        red[threadIdx.x] = t;
        __syncthreads();
        for (int off = 128; off > 0; off >>= 1) {
            if ((int)threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
            __syncthreads();
        }
        nu = nu_scale * red[0];
        if (threadIdx.x == 0) *nu_out = nu;
    }
    for (int e = threadIdx.x; e < ldo * ldo; e += blockDim.x) {
        const int i = e / ldo, j = e - i * ldo;
        float v = 0.f;
        if (i < l && j < l) v = 0.5f * (G[(size_t)i * ldg + j] + G[(size_t)j * ldg + i]) + (i == j ? nu : 0.f);
        if (out64) out64[e] = (double)v;
        else out[e] = v;
    }
}

// Y[i][c] += nu Q[i][c] for c < l (nu read from the device).
__global__ void __launch_bounds__(256)
add_scaled_kernel(float *__restrict__ Y, const float *__restrict__ Q, int64_t rows, int l, int lp,
                  const float *__restrict__ nu_p) {
    const float nu = *nu_p;
    const int64_t total = rows * (int64_t)lp;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
        if ((int)(e % lp) < l) Y[e] = fmaf(nu, Q[e], Y[e]);
}

// S[r] = max(sig[r]^2 - nu, 0): Section 3's Sigma = S^2 with the shift taken back.
__global__ void nystrom_values_kernel(float *__restrict__ S, const float *__restrict__ sig, int k,
                                      const float *__restrict__ nu_p) {
    const float nu = *nu_p;
    for (int r = threadIdx.x; r < k; r += blockDim.x) S[r] = fmaxf(fmaf(sig[r], sig[r], -nu), 0.f);
}

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
    // room for FP64 factors (RPCA_PREC_SMALL_FP64)
    L.racc0 = take((size_t)l * l * 8);
    L.racc1 = take((size_t)l * l * 8);
    L.r32 = take((size_t)l * l * 4);
    L.wfull = take(lp * gram_ld(l) * 4);
    L.zfull = take(lp * gram_ld(l) * 4);
    L.svd64 = take(small_svd64_doubles(l) * 8);
    L.wk = take(lp * L.kp * 4);
    L.zk = take(lp * L.kp * 4);
    L.sig = take(lp * 4);
    L.perm = take(lp * 4);
    L.rot = take(small_svd_rot_floats(l) * 4);
    L.zbuf = take(256);
    L.rinv_m = take(lp * lp * 4);
    L.flags = take(256);
    L.scal = take(256);
    L.cvec = take((size_t)n * 4);
    L.bias = take(lp * 4);
    L.bpart = take((size_t)centring_parts(n) * lp * 4);
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
    if ((o->precision & ~(RPCA_PREC_BF16X3 | RPCA_PREC_SMALL_FP64)) != 0) return RPCA_ERR_INVALID_ARG;
    if (renorm_kind(o->renorm) != RPCA_RENORM_CHOLQR && renorm_kind(o->renorm) != RPCA_RENORM_LU)
        return RPCA_ERR_INVALID_ARG;
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
    bool fp64 = false;        // l x l work in FP64 (the accumulated factors are doubles)
    template <class T> T *at(size_t off) const { return reinterpret_cast<T *>(ws + off); }
};

// Cholesky + inverse (+ accumulated factor) of a reduced Gram matrix, FP32 or FP64.
int chol_step(const Ctx &c, const float *G, float *rinv, const void *racc_in, void *racc_out, int *shifted_out,
              const int *skip) {
    if (c.fp64)
        return launch_chol64(G, c.L.l, c.L.lp, rinv, static_cast<const double *>(racc_in),
                             static_cast<double *>(racc_out), c.st, c.s, shifted_out, skip);
    return launch_chol_inv(G, c.L.l, c.L.lp, rinv, static_cast<const float *>(racc_in), static_cast<float *>(racc_out),
                           c.st, c.s, shifted_out, skip);
}

// SVD of R^T for the accumulated factor in racc0 (FP32 or FP64).
int small_svd_step(const Ctx &c, float *wk, float *zk, float *sig) {
    const Layout &L = c.L;
    if (c.fp64)
        return launch_small_svd64(c.at<double>(L.racc0), L.l, L.lp, L.k, L.kp, wk, zk, sig, c.at<float>(L.rot),
                                  c.at<float>(L.zbuf), c.at<int>(L.perm), c.at<float>(L.r32), c.at<float>(L.wfull),
                                  c.at<float>(L.zfull), c.at<double>(L.svd64), c.st, c.s);
    return launch_small_svd(c.at<float>(L.racc0), L.l, L.lp, L.k, L.kp, wk, zk, sig, c.at<float>(L.rot),
                            c.at<float>(L.zbuf), c.at<int>(L.perm), c.st, c.s);
}

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
    return chol_step(c, G, rinv, racc_in, racc_out, shifted_out, skip);
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
int renorm_m(const Ctx &c, bool raw, bool final_, const float **q, bool *pending, bool centred = false) {
    const Layout &L = c.L;
    float *y0 = c.at<float>(L.y0), *y1 = c.at<float>(L.y1);
    int *flag = c.at<int>(L.flags);
    if (!raw && !centred) {
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
                                   c.at<float>(L.qpart), L.cchunks, c.s, c.at<float>(L.cvec)));
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
          renorm_kind(o->renorm) == RPCA_RENORM_LU, small_fp64(o->precision)};
    op.scratch = reinterpret_cast<char *>(ws) + L.scratch;
    op.st = c.st;
    const bool raw = o->raw != 0;
    const bool odd_only = renorm_odd_only(o->renorm);
    const int l = L.l, lp = L.lp;
    float *x0 = c.at<float>(L.x0), *x1 = c.at<float>(L.x1), *y0 = c.at<float>(L.y0), *y1 = c.at<float>(L.y1);

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

    // Products with A.  Centring (Section 5: A*X - ones(m,1)*(c*X)): the sketch comes
    // before any adjoint product, so its rows are centred on their own mean (the mean of
    // the rows of A X is c X); after the first adjoint pass has produced c, the row
    // vector c X is formed from the small block and subtracted in the product's epilogue.
    const bool fuse = !raw && op.fuses_bias();
    float *bias = c.at<float>(L.bias);
    auto apply = [&](const float *X, bool with_bias) {
        if (with_bias) {
            TimedScope tc(kTimeCentre, s);
            RPCA_TRY(launch_centring_row(c.at<float>(L.cvec), X, L.n, l, lp, c.at<float>(L.bpart), bias, s));
        }
        TimedScope ts(kTimeApply, s);
        return op.apply(X, lp, y0, s, with_bias ? bias : nullptr);
    };
    // sketch and power iterations; odd-only: the products with A^* (the even-numbered
    // ones) feed the next product with A unrenormalised (x0's padding columns are zero)
    const float *q = nullptr;
    bool pending = false;
    RPCA_TRY(apply(x1, false));
    RPCA_TRY(renorm_m(c, raw, o->its == 0, &q, &pending));
    for (int it = 1; it <= o->its; ++it) {
        RPCA_TRY(adjoint_pass(op, c, raw, q, pending));
        if (!odd_only) RPCA_TRY(renorm_n(c, false));
        // the block that becomes the final Q is centred on its own row mean unless the
        // bias matches the product exactly (intermediate blocks reach the output only
        // through A_c^*, which annihilates the ones direction)
        const bool with_bias = fuse && (it < o->its || op.exact_bias(lp));
        RPCA_TRY(apply(odd_only ? x0 : x1, with_bias));
        RPCA_TRY(renorm_m(c, raw, it == o->its, &q, &pending, with_bias));
    }

    // B^* = A_c^* Q (Eq. i2), B^* = Q2 R, SVD of R^T (Eq. i3)
    RPCA_TRY(adjoint_pass(op, c, raw, q, pending));
    RPCA_TRY(renorm_n(c, true));
    float *wk = c.at<float>(L.wk), *zk = c.at<float>(L.zk), *sig = c.at<float>(L.sig);
    {
        TimedScope ts(kTimeSmallSvd, s);
        RPCA_TRY(small_svd_step(c, wk, zk, sig));
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

// Self-adjoint A (n x n, m == n in the layout).  Section 5's loop: Q = A Q each
// iteration, renormalised (LU or CholeskyQR) when it < its -- only in the odd
// iterations with RPCA_RENORM_ODD_ONLY -- and orthonormalised (CholeskyQR two or three
// times) when it == its.  Blocks ping-pong between y0 and x0 (both n x lp here);
// renormalised blocks go to x1, the final Q to y1.
int run_pipeline_sym(Operator &op, const rpca_opts *o, bool nystrom, float *U, int64_t ldu, float *S, float *V,
                     int64_t ldv, void *ws, const Layout &L, cudaStream_t s) {
    Ctx c{L, reinterpret_cast<char *>(ws), s, reinterpret_cast<DevStatus *>(reinterpret_cast<char *>(ws) + L.status),
          renorm_kind(o->renorm) == RPCA_RENORM_LU, small_fp64(o->precision)};
    op.scratch = reinterpret_cast<char *>(ws) + L.scratch;
    op.st = c.st;
    const bool odd_only = renorm_odd_only(o->renorm);
    const int l = L.l, lp = L.lp;
    const int64_t n = L.n;
    float *x0 = c.at<float>(L.x0), *x1 = c.at<float>(L.x1), *y0 = c.at<float>(L.y0), *y1 = c.at<float>(L.y1);
    float *nu = c.at<float>(L.scal);
    if (cudaMemsetAsync(c.st, 0, sizeof(DevStatus), s) != cudaSuccess) return RPCA_ERR_CUDA;
    if (cudaMemsetAsync(x1, 0, (size_t)n * lp * 4, s) != cudaSuccess) return RPCA_ERR_CUDA;
    if (o->omega) {
        const int64_t grid = std::min<int64_t>(cdiv(n * (int64_t)l, 256), (int64_t)num_sms() * 8);
        copy_scale_kernel<<<(unsigned)grid, 256, 0, s>>>(n, l, o->omega, l, o->col_weights, x1, lp);
        RPCA_CHECK_LAUNCH();
    } else {
        RPCA_TRY(launch_omega(n, l, o->seed, 0, o->col_weights, x1, lp, s));
    }
    auto apply = [&](const float *X, float *Y) {
        TimedScope ts(kTimeApply, s);
        return op.apply(X, lp, Y, s, nullptr);
    };
    const float *cur = x1;
    for (int it = 1; it <= o->its; ++it) {
        float *out = cur == y0 ? x0 : y0;
        RPCA_TRY(apply(cur, out));
        if (it == o->its) {
            int *flag = c.at<int>(L.flags);
            float *other = out == y0 ? x0 : y0;
            RPCA_TRY(cholqr_round(c, out, y1, n, L.s_gram_m, nullptr, nullptr, flag));
            RPCA_TRY(cholqr_round(c, y1, other, n, L.s_gram_m, nullptr, nullptr));
            RPCA_TRY(cholqr_round(c, other, y1, n, L.s_gram_m, nullptr, nullptr, nullptr, flag));
        } else if (!odd_only || it % 2 == 1) {
            if (c.lu) {
                float *rinv = c.at<float>(L.rinv);
                RPCA_TRY(lu_factor(c, out, n, rinv));
                TimedScope ts(kTimeTrsm, s);
                RPCA_TRY(launch_sgemm(false, n, lp, lp, out, lp, rinv, lp, x1, lp, 1, 0, s));
            } else {
                RPCA_TRY(cholqr_round(c, out, x1, n, L.s_gram_m, nullptr, nullptr));
            }
            cur = x1;
        } else {
            cur = out;
        }
    }
    RPCA_TRY(launch_finalize(y1, n, l, lp, 0.f, nullptr, s));

    // B = Q^T (A Q): split-K partials and their compensated reduction
    RPCA_TRY(apply(y1, y0));
    float *part = c.at<float>(L.part), *G = c.at<float>(L.G);
    {
        TimedScope ts(kTimeGram, s);
        RPCA_TRY(launch_sgemm(true, lp, lp, n, y1, lp, y0, lp, part, lp, L.s_gram_m, (int64_t)lp * lp, s));
        RPCA_TRY(launch_gram_reduce(part, L.s_gram_m, l, lp, G, s));
    }
    float *wk = c.at<float>(L.wk), *zk = c.at<float>(L.zk), *sig = c.at<float>(L.sig);
    float *racc0 = c.at<float>(L.racc0);
    if (!nystrom) {
        // symmetric B = W Sigma Z^T (Jacobi); U = Q W, V = Q Z (Eqs. i3, i4 with B = Q^T A Q)
        symmetrize_kernel<<<1, 256, 0, s>>>(G, l, gram_ld(l), racc0, l, 0.f, nullptr,
                                            c.fp64 ? c.at<double>(L.racc0) : nullptr);
        RPCA_CHECK_LAUNCH();
        {
            TimedScope ts(kTimeSmallSvd, s);
            RPCA_TRY(small_svd_step(c, wk, zk, sig));
        }
        TimedScope ts_lift(kTimeLift, s);
        RPCA_TRY(launch_sgemm(false, n, L.k, lp, y1, lp, zk, L.kp, V, ldv, 1, 0, s));
        RPCA_TRY(launch_sign_fix(V, n, ldv, L.k, wk, lp, L.kp, sig, S, s));
        return launch_sgemm(false, n, L.k, lp, y1, lp, wk, L.kp, U, ldu, 1, 0, s);
    }
    // Section 3 with A + nu I: B1 = A Q + nu Q, B2 = Q^T B1 = sym(Q^T A Q) + nu I,
    // C^T C = B2, F = B1 C^-1, F = Q2 R (CholeskyQR), R^T = W Sigma Z^T, so the left
    // singular vectors of F are Q2 Z and its singular values Sigma; S = Sigma^2 - nu.
    // nu = 2 (16 l + sqrt(n)) 2^-24 tr(B2): twice the FP32 Cholesky's collapse threshold
    // (16 l u of a diagonal entry) plus the rounding of the n-term products behind B2.
    float *B2 = c.at<float>(L.rinv_m);
    const float nu_scale = (float)(2.0 * (16.0 * l + std::sqrt((double)n)) * 0x1p-24);
    symmetrize_kernel<<<1, 256, 0, s>>>(G, l, gram_ld(l), B2, gram_ld(l), nu_scale, nu);
    RPCA_CHECK_LAUNCH();
    {
        const int64_t grid = std::min<int64_t>(cdiv(n * (int64_t)lp, 256), (int64_t)num_sms() * 8);
        add_scaled_kernel<<<(unsigned)grid, 256, 0, s>>>(y0, y1, n, l, lp, nu);
        RPCA_CHECK_LAUNCH();
    }
    float *rinv = c.at<float>(L.rinv);
    {
        TimedScope ts(kTimeChol, s);
        RPCA_TRY(chol_step(c, B2, rinv, nullptr, nullptr, nullptr, nullptr));
    }
    {
        TimedScope ts(kTimeTrsm, s);
        if (tc_rmul_ok(n, lp))
            RPCA_TRY(launch_tc_rmul(y0, n, lp, rinv, lp, lp, c.at<__nv_bfloat16>(L.rsplit), x0, lp, nullptr, c.st, s));
        else
            RPCA_TRY(launch_sgemm(false, n, lp, lp, y0, lp, rinv, lp, x0, lp, 1, 0, s));
    }
    RPCA_TRY(renorm_n(c, true));
    {
        TimedScope ts(kTimeSmallSvd, s);
        RPCA_TRY(small_svd_step(c, wk, zk, sig));
    }
    TimedScope ts_lift(kTimeLift, s);
    RPCA_TRY(launch_sgemm(false, n, L.k, lp, x1, lp, zk, L.kp, U, ldu, 1, 0, s));
    RPCA_TRY(launch_sign_fix(U, n, ldu, L.k, wk, lp, L.kp, sig, S, s));
    nystrom_values_kernel<<<1, 256, 0, s>>>(S, sig, L.k, nu);
    RPCA_CHECK_LAUNCH();
    return RPCA_OK;
}

}  // namespace rpca

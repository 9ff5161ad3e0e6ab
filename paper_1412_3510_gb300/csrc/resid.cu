// Spectral-norm residual ||A_c - U diag(S) V^T|| by the power method from a
// random start (Section 4; Kuczynski & Wozniakowski, Theorem 4.1(a): the
// estimate is within a factor of two with high probability).
//
// E = A_c - U S V^T is never formed.  Each iteration: t = V^T x;
// y = A x - mean(A x) - U (S t)   (centring as for every A-side product);
// t2 = U^T y;  z = A^T y - c (1^T y) - V (S t2)   (adjoint with the ones column);
// lambda = |z|, x = z / lambda.  The estimate sqrt(lambda) never exceeds ||E||.
// The products reuse the pipeline's operators with a block of width 8
// (x or y in column 0, the ones column in column 1).
#include "pipeline.cuh"
#include "resid.cuh"

namespace rpca {

namespace {

constexpr int kW = 8;            // block width of the GEMV-like products
constexpr int kRows = 512;       // rows per partial

// part[chunk * k + r] = sum over the chunk's rows i of M[i][r] * x[i * ldx]
__global__ void __launch_bounds__(256)
wcolsum_kernel(const float *__restrict__ M, int64_t rows, int k, int64_t ldm,
               const float *__restrict__ x, int64_t ldx, float *__restrict__ part) {
    __shared__ float red[256];
    const int64_t r0 = (int64_t)blockIdx.x * kRows, r1 = min(rows, r0 + kRows);
    for (int cb = 0; cb < k; cb += 32) {
        const int c = cb + (threadIdx.x & 31), g = threadIdx.x >> 5;   // 8 row groups
        float s = 0.f;
        if (c < k)
            for (int64_t i = r0 + g; i < r1; i += 8) s = fmaf(M[i * ldm + c], x[i * ldx], s);
        red[threadIdx.x] = s;
        __syncthreads();
        if (threadIdx.x < 32 && c < k) {
            float t = 0.f;
            for (int q = 0; q < 8; ++q) t += red[q * 32 + threadIdx.x];
            part[(int64_t)blockIdx.x * k + c] = t;
        }
        __syncthreads();
    }
}

__device__ void reduce_parts(const float *__restrict__ part, int chunks, int k,
                             const float *__restrict__ S, float *__restrict__ st_out) {
    for (int r = threadIdx.x; r < k; r += blockDim.x) {
        double s = 0.0;
        for (int q = 0; q < chunks; ++q) s += (double)part[(int64_t)q * k + r];
        st_out[r] = (float)s * S[r];
    }
}

// y_i = w_i - mean(w) - sum_r U[i][r] S[r] t[r]; Q8 row i = (y_i, ones, 0...);
// ypart[chunk] = sum of the chunk's y_i.
__global__ void __launch_bounds__(256)
combine_m_kernel(const float *__restrict__ W8, int64_t m, const float *__restrict__ wpart, int wchunks,
                 int centre, const float *__restrict__ U, int64_t ldu, const float *__restrict__ S,
                 const float *__restrict__ tpart, int tchunks, int k, float *__restrict__ Q8,
                 float *__restrict__ ypart) {
    __shared__ float st[RPCA_MAX_L];
    __shared__ float red[256];
    __shared__ float s_mean;
    reduce_parts(tpart, tchunks, k, S, st);
    if (threadIdx.x == 0) {
        double s = 0.0;
        if (centre)
            for (int q = 0; q < wchunks; ++q) s += (double)wpart[q];
        s_mean = (float)(s / (double)m);
    }
    __syncthreads();
    const int64_t r0 = (int64_t)blockIdx.x * kRows, r1 = min(m, r0 + kRows);
    float acc = 0.f;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        float y = W8[i * kW] - s_mean;
        const float *u = U + i * ldu;
        for (int r = 0; r < k; ++r) y = fmaf(-u[r], st[r], y);
        float *q = Q8 + i * kW;
        q[0] = y;
        q[1] = centre ? 1.f : 0.f;
#pragma unroll
        for (int c = 2; c < kW; ++c) q[c] = 0.f;
        acc += y;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int off = 128; off > 0; off >>= 1) {
        if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) ypart[blockIdx.x] = red[0];
}

// z_j = Z8[j][0] - sum_r V[j][r] S[r] t2[r]; X8[j][0] = z_j (unnormalised);
// npart[chunk] = sum of z_j^2 (FP64).
__global__ void __launch_bounds__(256)
combine_n_kernel(const float *__restrict__ Z8, int64_t n, const float *__restrict__ V, int64_t ldv,
                 const float *__restrict__ S, const float *__restrict__ t2part, int t2chunks, int k,
                 float *__restrict__ X8, double *__restrict__ npart) {
    __shared__ float st[RPCA_MAX_L];
    __shared__ double red[256];
    reduce_parts(t2part, t2chunks, k, S, st);
    __syncthreads();
    const int64_t r0 = (int64_t)blockIdx.x * kRows, r1 = min(n, r0 + kRows);
    double acc = 0.0;
    for (int64_t j = r0 + threadIdx.x; j < r1; j += blockDim.x) {
        float z = Z8[j * kW];
        const float *v = V + j * ldv;
        for (int r = 0; r < k; ++r) z = fmaf(-v[r], st[r], z);
        X8[j * kW] = z;
        acc += (double)z * (double)z;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int off = 128; off > 0; off >>= 1) {
        if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) npart[blockIdx.x] = red[0];
}

// lambda = sqrt(sum npart); X8[:,0] /= lambda; est = sqrt(lambda) when est != NULL.
__global__ void __launch_bounds__(256)
normalize_kernel(float *__restrict__ X8, int64_t n, const double *__restrict__ npart, int chunks,
                 double *__restrict__ est, int first) {
    __shared__ double s_lam;
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < chunks; ++q) s += npart[q];
        s_lam = sqrt(s);
    }
    __syncthreads();
    const double lam = s_lam;
    const float inv = lam > 0.0 ? (float)(1.0 / lam) : 0.f;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x)
        X8[j * kW] *= inv;
    // first call normalises the start vector (lambda = |x0|, no estimate)
    if (est && !first && blockIdx.x == 0 && threadIdx.x == 0) *est = sqrt(lam);
}

// npart[chunk] = sum over the chunk of X8[j][0]^2 (start vector).
__global__ void __launch_bounds__(256)
sumsq_kernel(const float *__restrict__ X8, int64_t n, double *__restrict__ npart) {
    __shared__ double red[256];
    const int64_t r0 = (int64_t)blockIdx.x * kRows, r1 = min(n, r0 + kRows);
    double acc = 0.0;
    for (int64_t j = r0 + threadIdx.x; j < r1; j += blockDim.x) {
        const double z = X8[j * kW];
        acc += z * z;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int off = 128; off > 0; off >>= 1) {
        if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) npart[blockIdx.x] = red[0];
}

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

ResidLayout make_resid_layout(int64_t m, int64_t n, int k, int adj_splits) {
    ResidLayout R;
    R.m = m; R.n = n; R.k = k; R.s_adj = std::max(adj_splits, 1);
    R.mchunks = (int)cdiv(m, kRows);
    R.nchunks = (int)cdiv(n, kRows);
    size_t off = 0;
    auto take = [&](size_t b) { const size_t o = off; off = a256(off + b); return o; };
    R.status = take(sizeof(DevStatus));
    R.x8 = take((size_t)n * kW * 4);
    R.z8 = take((size_t)n * kW * 4);
    R.w8 = take((size_t)m * kW * 4);
    R.q8 = take((size_t)m * kW * 4);
    R.part = take((size_t)R.s_adj * n * kW * 4);
    R.wpart = take((size_t)colsum_chunks(m) * 4);
    R.ypart = take((size_t)R.mchunks * 4);
    R.tpart = take((size_t)R.nchunks * std::max(k, 1) * 4);
    R.t2part = take((size_t)R.mchunks * std::max(k, 1) * 4);
    R.npart = take((size_t)R.nchunks * 8);
    R.total = off;
    return R;
}

int run_resid(const Operator &op, int raw, const float *U, int64_t ldu, const float *S, const float *V,
              int64_t ldv, int k, int iters, uint64_t seed, double *est, void *ws, const ResidLayout &R,
              cudaStream_t s, bool clear_status) {
    char *w = reinterpret_cast<char *>(ws);
    auto F = [&](size_t o) { return reinterpret_cast<float *>(w + o); };
    DevStatus *st = reinterpret_cast<DevStatus *>(w + R.status);
    float *x8 = F(R.x8), *z8 = F(R.z8), *w8 = F(R.w8), *q8 = F(R.q8), *part = F(R.part);
    float *wpart = F(R.wpart), *ypart = F(R.ypart), *tpart = F(R.tpart), *t2part = F(R.t2part);
    double *npart = reinterpret_cast<double *>(w + R.npart);
    const int64_t m = R.m, n = R.n;
    const int centre = raw ? 0 : 1;

    if (clear_status && cudaMemsetAsync(st, 0, sizeof(DevStatus), s) != cudaSuccess) return RPCA_ERR_CUDA;
    if (cudaMemsetAsync(x8, 0, (size_t)n * kW * 4, s) != cudaSuccess) return RPCA_ERR_CUDA;
    if (cudaMemsetAsync(est, 0, sizeof(double), s) != cudaSuccess) return RPCA_ERR_CUDA;
    RPCA_TRY(launch_omega(n, 1, seed, 1, nullptr, x8, kW, s));
    sumsq_kernel<<<R.nchunks, 256, 0, s>>>(x8, n, npart);
    RPCA_CHECK_LAUNCH();
    const int ngrid = (int)std::min<int64_t>(cdiv(n, 256), (int64_t)num_sms() * 4);
    normalize_kernel<<<ngrid, 256, 0, s>>>(x8, n, npart, R.nchunks, nullptr, 1);
    RPCA_CHECK_LAUNCH();

    for (int it = 0; it < iters; ++it) {
        if (k > 0) {
            wcolsum_kernel<<<R.nchunks, 256, 0, s>>>(V, n, k, ldv, x8, kW, tpart);
            RPCA_CHECK_LAUNCH();
        }
        RPCA_TRY(op.apply(x8, kW, w8, s, nullptr));
        int wch = 0;
        if (centre) RPCA_TRY(launch_colsum_partial(w8, m, 1, kW, wpart, &wch, s));
        combine_m_kernel<<<R.mchunks, 256, 0, s>>>(w8, m, wpart, wch, centre, U, ldu, S, tpart,
                                                   R.nchunks, k, q8, ypart);
        RPCA_CHECK_LAUNCH();
        if (k > 0) {
            wcolsum_kernel<<<R.mchunks, 256, 0, s>>>(U, m, k, ldu, q8, kW, t2part);
            RPCA_CHECK_LAUNCH();
        }
        RPCA_TRY(op.adjoint(q8, kW, part, s));
        RPCA_TRY(launch_adjoint_reduce(part, std::max(op.adjoint_splits(kW), 1), n, 1, kW, z8, centre,
                                       (double)m, ypart, R.mchunks, s));
        combine_n_kernel<<<R.nchunks, 256, 0, s>>>(z8, n, V, ldv, S, t2part, R.mchunks, k, x8, npart);
        RPCA_CHECK_LAUNCH();
        normalize_kernel<<<ngrid, 256, 0, s>>>(x8, n, npart, R.nchunks, est, 0);
        RPCA_CHECK_LAUNCH();
    }
    return RPCA_OK;
}

}  // namespace rpca

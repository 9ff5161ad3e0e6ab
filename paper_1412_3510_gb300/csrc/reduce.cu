// Column statistics and reductions around the products.
//
// Implicit centring (Section 5).  The paper applies the centred matrix as
// A*Q - ones(m,1)*(c*Q) with c the column means of A.  Since the means of the
// rows of A*Q are exactly c*Q, the A-side correction is applied here as
// "subtract from every row of Y = A*X the mean of Y's rows", which needs no
// separate pass over A.  The adjoint side, (Q'*A)' - c'*(ones(1,m)*Q), needs c
// itself: it arrives through a column of ones appended to Q (column l of the
// padded block), whose product with A^T is m c.
#include "internal.cuh"

#include <algorithm>

namespace rpca {

namespace {

constexpr int kChunkRows = 512;     // rows per partial column sum

// part[chunk * l + c] = sum of Y[r][c] over the rows r of the chunk (c < l).
// When write_pad, also set Y[r][l] = ones_value and Y[r][c] = 0 for l < c < ld.
__global__ void __launch_bounds__(256)
colsum_kernel(float *__restrict__ Y, int64_t rows, int l, int64_t ld, float *__restrict__ part,
              int write_pad, float ones_value) {
    __shared__ float red[256];
    const int64_t r0 = (int64_t)blockIdx.x * kChunkRows;
    const int64_t r1 = min(rows, r0 + kChunkRows);
    if (write_pad) {
        const int npad = (int)(ld - l);
        for (int64_t e = threadIdx.x; e < (r1 - r0) * npad; e += blockDim.x) {
            const int64_t r = r0 + e / npad;
            const int c = l + (int)(e % npad);
            Y[r * ld + c] = (c == l) ? ones_value : 0.f;
        }
    }
    if (!part) return;
    // 32 consecutive columns (coalesced rows) x 8 row groups, four independent sums
    // per thread; the eight group sums are combined in order
    __syncthreads();
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int cb = 0; cb < l; cb += 32) {
        const int c = cb + tx;
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
        if (c < l) {
            int64_t r = r0 + ty;
            for (; r + 24 < r1; r += 32) {
                s0 += Y[r * ld + c];
                s1 += Y[(r + 8) * ld + c];
                s2 += Y[(r + 16) * ld + c];
                s3 += Y[(r + 24) * ld + c];
            }
            for (; r < r1; r += 8) s0 += Y[r * ld + c];
        }
        red[threadIdx.x] = (s0 + s1) + (s2 + s3);
        __syncthreads();
        if (ty == 0 && c < l) {
            float tot = 0.f;
            for (int q = 0; q < 8; ++q) tot += red[q * 32 + tx];
            part[(int64_t)blockIdx.x * l + c] = tot;
        }
        __syncthreads();
    }
}

// One CTA: the column means (compensated FP32 sums of the partials, in chunk order)
// overwrite part[0 .. l) once every partial has been read.
__global__ void __launch_bounds__(256)
colmean_kernel(float *__restrict__ part, int64_t rows, int l, int nchunks) {
    __shared__ float mu[RPCA_MAX_L];
    for (int c = threadIdx.x; c < l; c += blockDim.x) {
        float s = 0.f, comp = 0.f;
        for (int q = 0; q < nchunks; ++q) {
            const float y = part[(int64_t)q * l + c] - comp;
            const float t = s + y;
            comp = (t - s) - y;
            s = t;
        }
        mu[c] = s / (float)rows;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < l; c += blockDim.x) part[c] = mu[c];
}

// Y[r][c] -= mu[c] (c < l), Y[r][c] = 0 (l <= c < ld).
__global__ void __launch_bounds__(256)
center_kernel(float *__restrict__ Y, int64_t rows, int l, int64_t ld, const float *__restrict__ mu_g) {
    __shared__ float mu[RPCA_MAX_L];
    const int tflat = threadIdx.y * blockDim.x + threadIdx.x;
    for (int c = tflat; c < l; c += blockDim.x * blockDim.y) mu[c] = mu_g[c];
    __syncthreads();
    // blockDim = (32, 8): threadIdx.x walks the columns of a row, threadIdx.y the rows
    for (int64_t r = blockIdx.x * (int64_t)blockDim.y + threadIdx.y; r < rows; r += (int64_t)gridDim.x * blockDim.y) {
        float *y = Y + r * ld;
        for (int c = threadIdx.x; c < ld; c += blockDim.x) y[c] = (c < l) ? y[c] - mu[c] : 0.f;
    }
}

// G[a][b] = sum_s part[s][a][b] (a, b < l), compensated (Kahan) FP32 sums in a
// fixed order: the result carries FP32-level relative error, as the FP32 Cholesky
// needs (GB300's FP64 adds run at 1/64 of the FP32 rate).  A CTA takes 32
// consecutive entries of G (threadIdx.x) and eight interleaved groups of the splits
// (threadIdx.y): every load is a coalesced 128-byte row of a partial, eight
// independent chains per entry; the eight group sums are combined in order.
__global__ void __launch_bounds__(256)
gram_reduce_kernel(const float *__restrict__ part, int splits, int l, int lp, float *__restrict__ G,
                   const int *__restrict__ skip_flag) {
    if (skip_flag && *skip_flag == 0) return;
    __shared__ float sh[8][32], ch[8][32];
    const int ldg = gram_ld(l);
    const int64_t total = (int64_t)ldg * ldg;
    const int64_t e = (int64_t)blockIdx.x * 32 + threadIdx.x;
    const int y = threadIdx.y;
    const int a = (int)(e / ldg), b = (int)(e % ldg);
    const bool in = e < total && a < l && b < l;
    float s = 0.f, comp = 0.f;
    if (in) {
        const float *p = part + (int64_t)a * lp + b;
        const int64_t stride = (int64_t)lp * lp;
        for (int q = y; q < splits; q += 8) {
            const float v = p[q * stride] - comp;
            const float t = s + v;
            comp = (t - s) - v;
            s = t;
        }
    }
    sh[y][threadIdx.x] = s;
    ch[y][threadIdx.x] = comp;
    __syncthreads();
    if (y == 0 && e < total) {
        float t = 0.f, c = 0.f;
        for (int g = 0; g < 8; ++g) {
            const float v = (sh[g][threadIdx.x] - ch[g][threadIdx.x]) - c;
            const float u = t + v;
            c = (u - t) - v;
            t = u;
        }
        G[e] = in ? t : 0.f;
    }
}

// X[j][c] = sum_s part[s][j][c]; centring: X[j][c] -= (X[j][l] / m) * qsum[c] (c < l);
// padding columns zeroed.  qsum[c] = sum of the Q column-sum partials.
__global__ void __launch_bounds__(256)
adjoint_reduce_kernel(const float *__restrict__ part, int splits, int64_t rows, int l, int lp,
                      float *__restrict__ X, int centre, float inv_m,
                      const float *__restrict__ qpart, int qchunks, float *__restrict__ cvec) {
    __shared__ float qsum[RPCA_MAX_L];
    if (centre) {
        for (int c = threadIdx.x; c < l; c += blockDim.x) {
            float s = 0.f, comp = 0.f;            // compensated sum of the partials
            for (int q = 0; q < qchunks; ++q) {
                const float y = qpart[(int64_t)q * l + c] - comp;
                const float t = s + y;
                comp = (t - s) - y;
                s = t;
            }
            qsum[c] = s;
        }
        __syncthreads();
    }
    const int64_t stride = rows * lp;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.y + threadIdx.y; j < rows;
         j += (int64_t)gridDim.x * blockDim.y) {
        const float *p = part + j * lp;
        float cj = 0.f;
        if (centre) {
            float s = 0.f;
            for (int q = 0; q < splits; ++q) s += p[q * stride + l];
            cj = s * inv_m;
            if (cvec && threadIdx.x == 0) cvec[j] = cj;
        }
        for (int c = threadIdx.x; c < lp; c += blockDim.x) {
            float v = 0.f;
            if (c < l) {
                float s = 0.f, comp = 0.f;
                for (int q = 0; q < splits; ++q) {
                    const float y = p[q * stride + c] - comp;
                    const float t = s + y;
                    comp = (t - s) - y;
                    s = t;
                }
                v = centre ? s - cj * qsum[c] : s;
            }
            X[j * lp + c] = v;
        }
    }
}

// bias[j] = sum_i c[i] X[i][j] (j < l), 0 for l <= j < lp, in two deterministic stages:
// CTA b sums the rows [b rows_per, (b + 1) rows_per) into part[b][j] (a warp reads 32
// consecutive columns of a row, eight warps take interleaved rows, the eight sums are
// combined in order), then one CTA adds the partials in CTA order (compensated).
constexpr int kCentreRowsPer = 64;
__global__ void __launch_bounds__(256)
centring_part_kernel(const float *__restrict__ c, const float *__restrict__ X, int64_t n, int l, int lp,
                     float *__restrict__ part) {
    __shared__ float sh[8][32];
    const int64_t r0 = (int64_t)blockIdx.x * kCentreRowsPer, r1 = min(n, r0 + kCentreRowsPer);
    const int y = threadIdx.y;
    for (int cb = 0; cb < lp; cb += 32) {
        const int j = cb + threadIdx.x;
        float acc = 0.f;
        if (j < l)
            for (int64_t i = r0 + y; i < r1; i += 8) acc = fmaf(c[i], X[i * lp + j], acc);
        sh[y][threadIdx.x] = acc;
        __syncthreads();
        if (y == 0 && j < lp) {
            float t = 0.f;
            for (int g = 0; g < 8; ++g) t += sh[g][threadIdx.x];
            part[(int64_t)blockIdx.x * lp + j] = t;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256)
centring_sum_kernel(const float *__restrict__ part, int nparts, int l, int lp, float *__restrict__ bias) {
    for (int j = threadIdx.x; j < lp; j += blockDim.x) {
        float s = 0.f, comp = 0.f;
        if (j < l)
            for (int b = 0; b < nparts; ++b) {
                const float v = part[(int64_t)b * lp + j] - comp;
                const float t = s + v;
                comp = (t - s) - v;
                s = t;
            }
        bias[j] = s;
    }
}

__global__ void fill_kernel(float *p, int64_t count, float value) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x)
        p[e] = value;
}

}  // namespace

int colsum_chunks(int64_t rows) { return (int)cdiv(std::max<int64_t>(rows, 1), kChunkRows); }

int launch_colsum_partial(const float *Y, int64_t rows, int l, int64_t ld, float *part,
                          int *nchunks, cudaStream_t s) {
    const int nc = colsum_chunks(rows);
    if (nchunks) *nchunks = nc;
    colsum_kernel<<<nc, 256, 0, s>>>(const_cast<float *>(Y), rows, l, ld, part, 0, 0.f);
    RPCA_CHECK_LAUNCH();
    return RPCA_OK;
}

int launch_finalize(float *Q, int64_t rows, int l, int64_t ld, float ones_value, float *part,
                    cudaStream_t s) {
    const int nc = colsum_chunks(rows);
    colsum_kernel<<<nc, 256, 0, s>>>(Q, rows, l, ld, part, 1, ones_value);
    RPCA_CHECK_LAUNCH();
    return RPCA_OK;
}

int launch_center(float *Y, int64_t rows, int l, int64_t ld, const float *part, int nchunks,
                  cudaStream_t s) {
    const int64_t grid = std::min<int64_t>(cdiv(rows, 8), (int64_t)num_sms() * 4);
    colmean_kernel<<<1, 256, 0, s>>>(const_cast<float *>(part), rows, l, nchunks);
    RPCA_CHECK_LAUNCH();
    center_kernel<<<(unsigned)std::max<int64_t>(grid, 1), dim3(32, 8), 0, s>>>(Y, rows, l, ld, part);
    RPCA_CHECK_LAUNCH();
    return RPCA_OK;
}

int launch_gram_reduce(const float *part, int splits, int l, int lp, float *G, cudaStream_t s,
                       const int *skip_flag) {
    const int64_t total = (int64_t)gram_ld(l) * gram_ld(l);
    gram_reduce_kernel<<<(unsigned)cdiv(total, (int64_t)32), dim3(32, 8), 0, s>>>(part, splits, l, lp, G, skip_flag);
    RPCA_CHECK_LAUNCH();
    return RPCA_OK;
}

int launch_adjoint_reduce(const float *part, int splits, int64_t rows, int l, int lp, float *X,
                          int centre, double m, const float *qpart, int qchunks, cudaStream_t s, float *cvec) {
    dim3 block(32, 8);
    const int64_t grid = std::min<int64_t>(cdiv(rows, 8), (int64_t)num_sms() * 8);
    adjoint_reduce_kernel<<<(unsigned)std::max<int64_t>(grid, 1), block, 0, s>>>(
        part, splits, rows, l, lp, X, centre, (float)(1.0 / m), qpart, qchunks, centre ? cvec : nullptr);
    RPCA_CHECK_LAUNCH();
    return RPCA_OK;
}

int centring_parts(int64_t n) { return (int)cdiv(std::max<int64_t>(n, 1), kCentreRowsPer); }

int launch_centring_row(const float *c, const float *X, int64_t n, int l, int lp, float *part, float *bias,
                        cudaStream_t s) {
    const int nb = centring_parts(n);
    centring_part_kernel<<<(unsigned)nb, dim3(32, 8), 0, s>>>(c, X, n, l, lp, part);
    RPCA_CHECK_LAUNCH();
    centring_sum_kernel<<<1, 256, 0, s>>>(part, nb, l, lp, bias);
    RPCA_CHECK_LAUNCH();
    return RPCA_OK;
}

int launch_fill(float *p, int64_t count, float value, cudaStream_t s) {
    if (count <= 0) return RPCA_OK;
    const int64_t grid = std::min<int64_t>(cdiv(count, 256), (int64_t)num_sms() * 8);
    fill_kernel<<<(unsigned)grid, 256, 0, s>>>(p, count, value);
    RPCA_CHECK_LAUNCH();
    return RPCA_OK;
}

}  // namespace rpca

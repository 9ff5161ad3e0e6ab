// Gram matrices G = Y^T Y of tall-skinny blocks (the CholeskyQR renormalisation
// of Section 5's "renormalise after every product").
//
// Split over row chunks; each CTA accumulates its chunk's partial Gram in
// registers.  A thread owns PPT 4x4 blocks (bi <= bj) of the upper triangle;
// rows are staged through shared memory 64 at a time, so per row and block a
// thread does two 16-byte shared loads and 16 FMAs.  The partials are summed
// in a fixed order by gram_reduce (deterministic).
#include "internal.cuh"

namespace rpca {

namespace {

constexpr int kRowsStage = 64;

// Thread layout: P = round_up(pairs, 32) threads per row group, RG row groups per
// CTA (narrow blocks have few pairs; the groups keep the CTA full).  Group g takes
// rows g, g + RG, ... of every stage and writes its own partial (split index
// blockIdx.x * RG + g), so the fixed-order reduction sums blocks x RG partials.
template <int PPT>
__global__ void gram_kernel(const float *__restrict__ Y, int64_t rows, int lp, int64_t rows_per_block, int RG,
                            float *__restrict__ part, const int *__restrict__ skip_flag) {
    if (skip_flag && *skip_flag == 0) return;
    extern __shared__ float ys[];                 // kRowsStage x lp
    const int nb = lp / 4;
    const int npairs = nb * (nb + 1) / 2;
    const int P = (int)blockDim.x / RG;
    const int pt = threadIdx.x % P, rg = threadIdx.x / P;
    int bi[PPT], bj[PPT];
    bool live[PPT];
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        int p = pt + q * P;
        live[q] = p < npairs;
        if (!live[q]) p = 0;
        // pair index p -> (i, j), i <= j, row-major over the upper triangle
        int i = 0;
        while (p >= nb - i) { p -= nb - i; ++i; }
        bi[q] = i;
        bj[q] = i + p;
    }
    float acc[PPT][4][4];
#pragma unroll
    for (int q = 0; q < PPT; ++q)
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[q][a][b] = 0.f;

    const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
    const int64_t r1 = min(rows, r0 + rows_per_block);
    for (int64_t rb = r0; rb < r1; rb += kRowsStage) {
        const int nr = (int)min((int64_t)kRowsStage, r1 - rb);
        __syncthreads();
        const int n4 = nr * lp / 4;
        for (int e = threadIdx.x; e < n4; e += blockDim.x)
            reinterpret_cast<float4 *>(ys)[e] = __ldg(reinterpret_cast<const float4 *>(Y + rb * lp) + e);
        __syncthreads();
        for (int r = rg; r < nr; r += RG) {
            const float *row = ys + r * lp;
#pragma unroll
            for (int q = 0; q < PPT; ++q) {
                if (!live[q]) continue;
                const float4 a = *reinterpret_cast<const float4 *>(row + 4 * bi[q]);
                const float4 b = *reinterpret_cast<const float4 *>(row + 4 * bj[q]);
                const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
                for (int x = 0; x < 4; ++x)
#pragma unroll
                    for (int y = 0; y < 4; ++y) acc[q][x][y] = fmaf(av[x], bv[y], acc[q][x][y]);
            }
        }
    }
    float *out = part + ((int64_t)blockIdx.x * RG + rg) * lp * lp;
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        if (!live[q]) continue;
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) {
                const int a = 4 * bi[q] + x, b = 4 * bj[q] + y;
                out[(int64_t)a * lp + b] = acc[q][x][y];
                out[(int64_t)b * lp + a] = acc[q][x][y];
            }
    }
}

// row groups per CTA for a block of width lp
int gram_groups(int lp) {
    const int nb = lp / 4;
    const int P = (int)round_up(nb * (nb + 1) / 2, 32);
    int rg = 1;
    while (rg < 8 && P * rg * 2 <= 256) rg *= 2;
    return rg;
}

}  // namespace

int gram_splits(int64_t rows, int lp) {
    // partials = CTAs x row groups; short blocks: one 64-row stage per CTA, so that
    // the few thousand rows of an n-side block still spread over many SMs
    const int rg = gram_groups(lp);
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(cdiv(rows, kRowsStage), 4LL * num_sms()));
    return (int)(blocks * rg);
}

int launch_gram(const float *Y, int64_t rows, int lp, float *part, int splits, const int *skip_flag,
                cudaStream_t s) {
    const int nb = lp / 4;
    const int npairs = nb * (nb + 1) / 2;
    const int rg = gram_groups(lp);
    if (splits % rg) return RPCA_ERR_INVALID_ARG;
    const int blocks = splits / rg;
    const int64_t per = cdiv(std::max<int64_t>(rows, 1), blocks);
    const size_t smem = (size_t)kRowsStage * lp * sizeof(float);
    const int P = (int)std::min<int64_t>(512, round_up(npairs, 32));
    const int threads = P * rg;
    const int ppt = (int)cdiv(npairs, P);
    for (auto k : {gram_kernel<1>, gram_kernel<2>, gram_kernel<4>})
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)((size_t)kRowsStage * (RPCA_MAX_L + 16) * sizeof(float))) != cudaSuccess)
            return RPCA_ERR_CUDA;
    if (ppt <= 1) {
        gram_kernel<1><<<blocks, threads, smem, s>>>(Y, rows, lp, per, rg, part, skip_flag);
    } else if (ppt <= 2) {
        gram_kernel<2><<<blocks, threads, smem, s>>>(Y, rows, lp, per, rg, part, skip_flag);
    } else if (ppt <= 4) {
        gram_kernel<4><<<blocks, threads, smem, s>>>(Y, rows, lp, per, rg, part, skip_flag);
    } else {
        return RPCA_ERR_INVALID_ARG;
    }
    RPCA_CHECK_LAUNCH();
    return RPCA_OK;
}

}  // namespace rpca

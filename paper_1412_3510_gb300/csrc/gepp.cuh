// Partial-pivoting elimination of a small block held in shared memory by one CTA
// (the LU renormalisation of Section 5, used by the tall-skinny LU).
#pragma once

#include <cstdint>

namespace rpca {

struct GeppScratch {
    float wval[32];
    int warg[32];
    int piv;
};

// Eliminates the first l columns of M (nrows x ld, row r present when ids[r] >= 0):
// step j swaps the present row r >= j with the largest |M[r][j]| (the first on ties)
// into row j (rows of M and ids), then M[i][c] -= M[i][j] / M[j][j] * M[j][c] for
// i > j, c > j (skipped when M[j][j] == 0).  Afterwards ids[0 .. steps) are the pivot
// rows in pivot order and the upper triangle of M's first `steps` rows is U.
// Returns steps (< min(l, nrows) when the present rows run out).  All threads call it.
__device__ inline int gepp_block(float *M, int ld, int *ids, int nrows, int l, GeppScratch &g) {
    const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, lane = tid & 31, nwarps = nt >> 5;
    const int steps = min(l, nrows);
    int j = 0;
    for (; j < steps; ++j) {
        float best = -1.f;
        int arg = -1;
        for (int r = j + tid; r < nrows; r += nt) {
            if (ids[r] < 0) continue;
            const float v = fabsf(M[r * ld + j]);
            if (v > best) { best = v; arg = r; }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const float ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oa = __shfl_xor_sync(0xffffffffu, arg, o);
            if (ob > best || (ob == best && oa >= 0 && (arg < 0 || oa < arg))) { best = ob; arg = oa; }
        }
        if (lane == 0) { g.wval[warp] = best; g.warg[warp] = arg; }
        __syncthreads();
        if (tid == 0) {
            float b = -1.f;
            int a = -1;
            for (int w = 0; w < nwarps; ++w)
                if (g.warg[w] >= 0 && (g.wval[w] > b || (g.wval[w] == b && g.warg[w] < a))) { b = g.wval[w]; a = g.warg[w]; }
            g.piv = a;
        }
        __syncthreads();
        const int p = g.piv;
        if (p < 0) break;                                 // no rows left (uniform)
        if (p != j) {
            for (int c = tid; c < l; c += nt) {
                const float t = M[j * ld + c];
                M[j * ld + c] = M[p * ld + c];
                M[p * ld + c] = t;
            }
            if (tid == 0) { const int t = ids[j]; ids[j] = ids[p]; ids[p] = t; }
        }
        __syncthreads();
        const float d = M[j * ld + j];
        const int w = l - j - 1;
        if (d != 0.f && w > 0) {
            const float inv_d = 1.0f / d;
            for (int e = tid; e < (nrows - j - 1) * w; e += nt) {
                const int i = j + 1 + e / w, c = j + 1 + e % w;
                M[i * ld + c] = fmaf(-(M[i * ld + j] * inv_d), M[j * ld + c], M[i * ld + c]);
            }
        }
        __syncthreads();
    }
    return j;
}

}  // namespace rpca

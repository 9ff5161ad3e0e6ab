// Counter-based Philox4x64-10 (Salmon, Moraes, Dror & Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC'11) and the Box-Muller transform, shared by
// every kernel that draws Gaussian test vectors.  The stream keyed (seed, id)
// maps element e of a row-major rows x cols draw to output t = e % 4 of
// counter block e / 4; outputs (0,1) and (2,3) are the two Box-Muller pairs.
#pragma once

#include <cstdint>

namespace rpca {

__device__ __forceinline__ void philox4x64_10(uint64_t c0, uint64_t k0, uint64_t k1, uint64_t (&w)[4]) {
    constexpr uint64_t kM0 = 0xD2E7470EE14C6C93ull;   // multipliers
    constexpr uint64_t kM1 = 0xCA5A826395121157ull;
    constexpr uint64_t kW0 = 0x9E3779B97F4A7C15ull;   // Weyl key increments
    constexpr uint64_t kW1 = 0xBB67AE8584CAA73Bull;
    uint64_t c1 = 0, c2 = 0, c3 = 0;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += kW0; k1 += kW1; }
        const uint64_t hi0 = __umul64hi(kM0, c0), lo0 = kM0 * c0;
        const uint64_t hi1 = __umul64hi(kM1, c2), lo1 = kM1 * c2;
        const uint64_t n0 = hi1 ^ c1 ^ k0;
        const uint64_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    w[0] = c0; w[1] = c1; w[2] = c2; w[3] = c3;
}

// (top 23 bits + 1/2) / 2^23: exact in FP32, strictly inside (0, 1).
__device__ __forceinline__ float uniform23(uint64_t w) {
    return ((float)(uint32_t)(w >> 41) + 0.5f) * 0x1p-23f;
}

// Four N(0,1) values of counter block b of the stream (k0, k1).
__device__ __forceinline__ void gauss4(uint64_t b, uint64_t k0, uint64_t k1, float (&z)[4]) {
    uint64_t w[4];
    philox4x64_10(b, k0, k1, w);
    float sn, cs;
    float r = sqrtf(-2.0f * logf(uniform23(w[0])));
    sincospif(2.0f * uniform23(w[1]), &sn, &cs);
    z[0] = r * cs; z[1] = r * sn;
    r = sqrtf(-2.0f * logf(uniform23(w[2])));
    sincospif(2.0f * uniform23(w[3]), &sn, &cs);
    z[2] = r * cs; z[3] = r * sn;
}

}  // namespace rpca

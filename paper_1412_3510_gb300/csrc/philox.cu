// Test matrix of the sketch (Section 2: i.i.d. N(0,1) test vectors; Section 5
// notes that any fast i.i.d. law works).  Counter-based Philox4x64-10 from
// Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as easy as 1, 2, 3"
// (SC'11), followed by the Box-Muller transform in FP32.
#include "internal.cuh"

namespace rpca {

namespace {

constexpr uint64_t kM0 = 0xD2E7470EE14C6C93ull;   // Philox4x64 multipliers
constexpr uint64_t kM1 = 0xCA5A826395121157ull;
constexpr uint64_t kW0 = 0x9E3779B97F4A7C15ull;   // Weyl key increments
constexpr uint64_t kW1 = 0xBB67AE8584CAA73Bull;

struct Block4 { uint64_t w[4]; };

__device__ __forceinline__ Block4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2,
                                                uint64_t c3, uint64_t k0, uint64_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += kW0; k1 += kW1; }
        const uint64_t hi0 = __umul64hi(kM0, c0), lo0 = kM0 * c0;
        const uint64_t hi1 = __umul64hi(kM1, c2), lo1 = kM1 * c2;
        const uint64_t n0 = hi1 ^ c1 ^ k0;
        const uint64_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    Block4 b;
    b.w[0] = c0; b.w[1] = c1; b.w[2] = c2; b.w[3] = c3;
    return b;
}

// (top 23 bits + 1/2) / 2^23: exact in FP32, strictly inside (0, 1).
__device__ __forceinline__ float uniform23(uint64_t w) {
    return ((float)(uint32_t)(w >> 41) + 0.5f) * 0x1p-23f;
}

__global__ void omega_kernel(int64_t n, int l, uint64_t seed, uint64_t stream_id,
                             const float *__restrict__ weights, float *__restrict__ out,
                             int64_t ldo) {
    const int64_t total = n * (int64_t)l;
    const int64_t nblk = (total + 3) / 4;
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nblk;
         b += (int64_t)gridDim.x * blockDim.x) {
        const Block4 x = philox4x64_10((uint64_t)b, 0, 0, 0, seed, stream_id);
        float z[4];
        {
            const float r = sqrtf(-2.0f * logf(uniform23(x.w[0])));
            float sn, cs;
            sincospif(2.0f * uniform23(x.w[1]), &sn, &cs);
            z[0] = r * cs; z[1] = r * sn;
        }
        {
            const float r = sqrtf(-2.0f * logf(uniform23(x.w[2])));
            float sn, cs;
            sincospif(2.0f * uniform23(x.w[3]), &sn, &cs);
            z[2] = r * cs; z[3] = r * sn;
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int64_t e = 4 * b + t;
            if (e < total) {
                const int64_t i = e / l;
                const int j = (int)(e - i * l);
                float v = z[t];
                if (weights) v *= weights[i];
                out[i * ldo + j] = v;
            }
        }
    }
}

__global__ void philox_raw_kernel(uint64_t k0, uint64_t k1, uint64_t first, int64_t nblocks,
                                  uint64_t *__restrict__ out) {
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nblocks;
         b += (int64_t)gridDim.x * blockDim.x) {
        const Block4 x = philox4x64_10(first + (uint64_t)b, 0, 0, 0, k0, k1);
#pragma unroll
        for (int t = 0; t < 4; ++t) out[4 * b + t] = x.w[t];
    }
}

}  // namespace

int launch_omega(int64_t n, int l, uint64_t seed, uint64_t stream_id, const float *weights,
                 float *out, int64_t ldo, cudaStream_t s) {
    const int64_t nblk = (n * (int64_t)l + 3) / 4;
    if (nblk == 0) return RPCA_OK;
    const int threads = 256;
    const int64_t grid = std::min<int64_t>(cdiv(nblk, threads), (int64_t)num_sms() * 8);
    omega_kernel<<<(unsigned)grid, threads, 0, s>>>(n, l, seed, stream_id, weights, out, ldo);
    RPCA_CHECK_LAUNCH();
    return RPCA_OK;
}

}  // namespace rpca

extern "C" int rpca_gaussian_omega(int64_t n, int32_t l, uint64_t seed, uint64_t stream_id,
                                   float *omega, int64_t ldo, rpca_stream_t stream) {
    if (n < 0 || l < 1 || ldo < l || (!omega && n > 0)) return RPCA_ERR_INVALID_ARG;
    return rpca::launch_omega(n, l, seed, stream_id, nullptr, omega, ldo, (cudaStream_t)stream);
}

extern "C" int rpca_philox4x64_10(uint64_t key0, uint64_t key1, uint64_t first, int64_t nblocks,
                                  uint64_t *out, rpca_stream_t stream) {
    if (nblocks < 0 || (!out && nblocks > 0)) return RPCA_ERR_INVALID_ARG;
    if (nblocks == 0) return RPCA_OK;
    const int threads = 256;
    const int64_t grid = std::min<int64_t>(rpca::cdiv(nblocks, threads), (int64_t)rpca::num_sms() * 8);
    rpca::philox_raw_kernel<<<(unsigned)grid, threads, 0, (cudaStream_t)stream>>>(key0, key1, first,
                                                                                 nblocks, out);
    RPCA_CHECK_LAUNCH();
    return RPCA_OK;
}

// Test matrix of the sketch (Section 2: i.i.d. N(0,1) test vectors; Section 5
// notes that any fast i.i.d. law works).  Counter-based Philox4x64-10 from
// Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as easy as 1, 2, 3"
// (SC'11), followed by the Box-Muller transform in FP32.
#include "internal.cuh"
#include "philox.cuh"

namespace rpca {

namespace {

__global__ void omega_kernel(int64_t n, int l, uint64_t seed, uint64_t stream_id,
                             const float *__restrict__ weights, float *__restrict__ out,
                             int64_t ldo) {
    const int64_t total = n * (int64_t)l;
    const int64_t nblk = (total + 3) / 4;
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nblk;
         b += (int64_t)gridDim.x * blockDim.x) {
        float z[4];
        gauss4((uint64_t)b, seed, stream_id, z);
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
        uint64_t w[4];
        philox4x64_10(first + (uint64_t)b, k0, k1, w);
#pragma unroll
        for (int t = 0; t < 4; ++t) out[4 * b + t] = w[t];
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

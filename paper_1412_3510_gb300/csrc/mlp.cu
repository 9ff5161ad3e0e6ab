// Learned column weighting of the test matrix.
//
// Section 2 draws the test matrix with i.i.d. Gaussian entries and Section 5
// notes that the method does not depend on the exact law of those entries.
// The learned variant scales row j of Omega by d_j > 0, predicted from
// statistics of column j of A by a small MLP 16 -> 128 -> 128 -> 1 (ReLU),
// d_j = clip(exp(y_j), 1e-2, 1e2); the network is trained to output the log
// of the relative leverage n |V_k[j, :]|^2 / k of the column.
//
// Kernels here:
//   mlp_pack_kernel     FP32 parameters -> BF16 weights in the MMA's canonical
//                       K-major layout + FP32 biases (one device blob)
//   mlp_fwd_kernel      inference on the tcgen05 tensor cores: per 128 columns
//                       one M=128,N=128,K=16 MMA (layer 1), bias+ReLU in the
//                       epilogue written back as the next BF16 A operand, eight
//                       K=16 MMAs (layer 2), then bias+ReLU and the dot with w3
//                       in the epilogue; FP32 accumulators in tensor memory
//   mlp_grad_kernel     training: FP32 forward + backward of 64 samples per
//                       CTA in shared memory, per-CTA partial gradients
//   mlp_grad_reduce     fixed-order sum of the partials (deterministic)
//   mlp_adam_kernel     Adam (Kingma & Ba 2015) with bias correction
//   leverage_kernel     training labels t_j = log(n |V_k[j, :]|^2 / k + 1e-3)
#include "internal.cuh"
#include "tc_ptx.cuh"

#include <cuda_bf16.h>

namespace rpca {

namespace {

using namespace ptx;

constexpr int kF = RPCA_MLP_FEATURES;         // 16
constexpr int kH = RPCA_MLP_HIDDEN;           // 128
// parameter offsets (FP32, oracle order): W1 [F][H], b1, W2 [H][H], b2, w3, b3
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kF * kH;
constexpr int kOffW2 = kOffB1 + kH;
constexpr int kOffB2 = kOffW2 + kH * kH;
constexpr int kOffW3 = kOffB2 + kH;
constexpr int kOffB3 = kOffW3 + kH;
static_assert(kOffB3 + 1 == RPCA_MLP_PARAMS, "parameter count");
// packed blob (bytes): W1^T BF16 (H x F, K-major), W2^T BF16 (H x H, K-major), then
// FP32 b1, b2, w3, b3 and 3 pad floats
constexpr uint32_t kPW1 = 0;
constexpr uint32_t kPW2 = kPW1 + kH * kF * 2;                 // 4096
constexpr uint32_t kPBias = kPW2 + kH * kH * 2;               // 36864
constexpr uint32_t kBiasFloats = 3 * kH + 4;
static_assert(kPBias + kBiasFloats * 4 == RPCA_MLP_PACKED_BYTES, "packed size");

// byte offset of element (row, k) in a K-major no-swizzle tile of K columns:
// 8 x 16-byte core matrices, LBO = 128 B along K, SBO = (K / 8) * 128 B per 8 rows
__host__ __device__ constexpr uint32_t kmajor_off(int row, int k, int K) {
    return (uint32_t)((row >> 3) * (K / 8) * 128 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

__global__ void mlp_pack_kernel(const float *__restrict__ p, uint8_t *__restrict__ out) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int stride = gridDim.x * blockDim.x;
    for (int e = tid; e < kH * kF; e += stride) {       // (h, f) <- W1[f][h]
        const int h = e / kF, f = e % kF;
        *reinterpret_cast<__nv_bfloat16 *>(out + kPW1 + kmajor_off(h, f, kF)) =
            __float2bfloat16_rn(p[kOffW1 + f * kH + h]);
    }
    for (int e = tid; e < kH * kH; e += stride) {       // (n, k) <- W2[k][n]
        const int n = e / kH, k = e % kH;
        *reinterpret_cast<__nv_bfloat16 *>(out + kPW2 + kmajor_off(n, k, kH)) =
            __float2bfloat16_rn(p[kOffW2 + k * kH + n]);
    }
    float *bias = reinterpret_cast<float *>(out + kPBias);
    for (int e = tid; e < (int)kBiasFloats; e += stride) {
        float v = 0.f;
        if (e < kH) v = p[kOffB1 + e];
        else if (e < 2 * kH) v = p[kOffB2 + e - kH];
        else if (e < 3 * kH) v = p[kOffW3 + e - 2 * kH];
        else if (e == 3 * kH) v = p[kOffB3];
        bias[e] = v;
    }
}

// ---------------------------------------------------------------------------
// inference (tcgen05)
// ---------------------------------------------------------------------------
constexpr int kFwdThreads = 128;
constexpr uint32_t kSA1 = kPBias;                 // layer-1 A tile: 128 x 16 BF16
constexpr uint32_t kSA2 = kSA1 + 128 * kF * 2;    // layer-2 A tile: 128 x 128 BF16
constexpr uint32_t kSBias = kSA2 + 128 * kH * 2;
constexpr uint32_t kSBar = kSBias + kBiasFloats * 4 + 16;
constexpr uint32_t kFwdSmem = kSBar + 64 + 1024;  // + alignment slack
constexpr uint32_t kTmemCols = 256;               // two 128-column accumulators

__global__ void __launch_bounds__(kFwdThreads) mlp_fwd_kernel(const uint8_t *__restrict__ packed,
                                                              const float *__restrict__ F, int64_t N,
                                                              float *__restrict__ y, float *__restrict__ d,
                                                              DevStatus *st) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + kSBar);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + kSBar + 8);
    const float *bias = reinterpret_cast<const float *>(smem + kSBias);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // weights: W1^T | W2^T to the front, biases after the two A tiles
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(packed);
        constexpr int nw = (int)(kPBias / 16), nb = (int)(kBiasFloats * 4 / 16);
        for (int e = tid; e < nw + nb; e += kFwdThreads) {
            const uint4 v = src[e];
            if (e < nw) reinterpret_cast<uint4 *>(smem)[e] = v;
            else reinterpret_cast<uint4 *>(smem + kSBias)[e - nw] = v;
        }
    }
    if (tid == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
    const uint32_t a1 = smem_u32(smem + kSA1), a2 = smem_u32(smem + kSA2);
    const uint32_t w1 = smem_u32(smem + kPW1), w2 = smem_u32(smem + kPW2);
    const uint32_t idesc = instr_desc_bf16(128, kH);
    const int64_t ntiles = (N + 127) / 128;
    uint32_t phase = 0;
    volatile int never = 0;        // no external abort for this kernel
    bool ok = true;

    for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const int64_t j = t * 128 + tid;
        // layer-1 A operand: this thread's feature row in BF16
        {
            float f[kF];
#pragma unroll
            for (int c = 0; c < kF; ++c) f[c] = j < N ? F[j * kF + c] : 0.f;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                uint32_t w[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    __nv_bfloat162 b = __float22bfloat162_rn(make_float2(f[8 * h + 2 * e], f[8 * h + 2 * e + 1]));
                    w[e] = bf2_bits(b);
                }
                *reinterpret_cast<uint4 *>(smem + kSA1 + kmajor_off(tid, 8 * h, kF)) = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            umma_bf16(tmem, smem_desc(a1, 128, (kF / 8) * 128), smem_desc(w1, 128, (kF / 8) * 128), idesc, 0u);
            umma_commit(bar);
        }
        ok = __syncthreads_and(mbar_wait(bar, phase, &never));
        phase ^= 1;
        if (!ok) break;
        tc_fence_after();
        // epilogue 1: h1 = relu(z1 + b1) -> BF16 layer-2 A operand (row = tid)
#pragma unroll 1
        for (int c0 = 0; c0 < kH; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + lane_off + (uint32_t)c0, v);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                uint32_t w[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int c = c0 + 8 * h + 2 * e;
                    const float x0 = fmaxf(v[8 * h + 2 * e] + bias[c], 0.f);
                    const float x1 = fmaxf(v[8 * h + 2 * e + 1] + bias[c + 1], 0.f);
                    w[e] = bf2_bits(__float22bfloat162_rn(make_float2(x0, x1)));
                }
                *reinterpret_cast<uint4 *>(smem + kSA2 + kmajor_off(tid, c0 + 8 * h, kH)) =
                    make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int kk = 0; kk < kH / 16; ++kk)
                umma_bf16(tmem + kH, smem_desc(a2 + kk * 256, 128, (kH / 8) * 128),
                          smem_desc(w2 + kk * 256, 128, (kH / 8) * 128), idesc, kk > 0 ? 1u : 0u);
            umma_commit(bar);
        }
        ok = __syncthreads_and(mbar_wait(bar, phase, &never));
        phase ^= 1;
        if (!ok) break;
        tc_fence_after();
        // epilogue 2: y = w3 . relu(z2 + b2) + b3
        float acc = 0.f;
#pragma unroll 1
        for (int c0 = 0; c0 < kH; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + kH + lane_off + (uint32_t)c0, v);
#pragma unroll
            for (int e = 0; e < 16; ++e) acc = fmaf(bias[2 * kH + c0 + e], fmaxf(v[e] + bias[kH + c0 + e], 0.f), acc);
        }
        const float yv = acc + bias[3 * kH];
        if (j < N) {
            if (y) y[j] = yv;
            if (d) d[j] = fminf(fmaxf(expf(yv), 1e-2f), 1e2f);
        }
        tc_fence_before();
        __syncthreads();
    }
    if (!ok && tid == 0) {
        atomicAdd(&st->timeouts, 1);
        dev_fail(st, RPCA_ERR_TIMEOUT);
        // give an MMA that may still be in flight time to finish before TMEM is freed
        const long long t0 = clock64();
        while (clock64() - t0 < kWaitCycles / 100) {}
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

// ---------------------------------------------------------------------------
// training (FP32, shared memory)
// ---------------------------------------------------------------------------
constexpr int kS = 64;                 // samples per CTA
constexpr int kGradThreads = 256;
constexpr int kLdF = kF + 1, kLdH = kH + 1;   // odd strides: row and column reads conflict-free
struct GradSmem {
    float W1[kF * kH];
    float W2[kH * kLdH];
    float Fs[kS * kLdF];
    float H1[kS * kLdH];      // h1, later dz1
    float H2[kS * kLdH];      // h2, later dz2
    float b1[kH], b2[kH], w3[kH];
    float dy[kS];
    float red[kGradThreads / 32];
};

// C(i, j) = sum_k op(A)(i, k) op(B)(k, j) over shared-memory operands, one output per
// thread and step; epi(i, j, value) consumes it.  A warp shares i, so op(A) reads
// broadcast and op(B) reads hit 32 different banks (odd leading dimensions).
template <bool TA, bool TB, class Epi>
__device__ __forceinline__ void smem_mm(int M, int Nn, int K, const float *A, int lda, const float *B, int ldb,
                                        Epi epi) {
    for (int idx = threadIdx.x; idx < M * Nn; idx += blockDim.x) {
        const int i = idx / Nn, j = idx - i * Nn;
        float acc = 0.f;
        for (int k = 0; k < K; ++k)
            acc = fmaf(TA ? A[k * lda + i] : A[i * lda + k], TB ? B[j * ldb + k] : B[k * ldb + j], acc);
        epi(i, j, acc);
    }
}

__global__ void __launch_bounds__(kGradThreads) mlp_grad_kernel(const float *__restrict__ p,
                                                                const float *__restrict__ F,
                                                                const float *__restrict__ t, int64_t N,
                                                                float *__restrict__ part) {
    extern __shared__ float4 smem_f4[];
    GradSmem &sm = *reinterpret_cast<GradSmem *>(smem_f4);
    const int tid = threadIdx.x;
    const int64_t s0 = (int64_t)blockIdx.x * kS;
    const int ns = (int)(N - s0 < kS ? N - s0 : kS);
    float *out = part + (int64_t)blockIdx.x * (RPCA_MLP_PARAMS + 1);

    for (int e = tid; e < kF * kH; e += kGradThreads) sm.W1[e] = p[kOffW1 + e];
    for (int e = tid; e < kH * kH; e += kGradThreads) sm.W2[(e / kH) * kLdH + e % kH] = p[kOffW2 + e];
    for (int e = tid; e < kH; e += kGradThreads) {
        sm.b1[e] = p[kOffB1 + e];
        sm.b2[e] = p[kOffB2 + e];
        sm.w3[e] = p[kOffW3 + e];
    }
    for (int e = tid; e < kS * kF; e += kGradThreads) {
        const int s = e / kF, f = e % kF;
        sm.Fs[s * kLdF + f] = s < ns ? F[(s0 + s) * kF + f] : 0.f;
    }
    __syncthreads();
    // forward: h1 = relu(F W1 + b1), h2 = relu(h1 W2 + b2)
    smem_mm<false, false>(ns, kH, kF, sm.Fs, kLdF, sm.W1, kH,
                          [&](int i, int j, float v) { sm.H1[i * kLdH + j] = fmaxf(v + sm.b1[j], 0.f); });
    __syncthreads();
    smem_mm<false, false>(ns, kH, kH, sm.H1, kLdH, sm.W2, kLdH,
                          [&](int i, int j, float v) { sm.H2[i * kLdH + j] = fmaxf(v + sm.b2[j], 0.f); });
    __syncthreads();
    // y = h2 w3 + b3; residual r = y - t; dL/dy = 2 r / N; loss partial = sum r^2
    const float b3 = p[kOffB3];
    const int warp = tid >> 5, lane = tid & 31;
    float lsum = 0.f;
    for (int s = warp; s < ns; s += kGradThreads / 32) {
        float a = 0.f;
        for (int h = lane; h < kH; h += 32) a = fmaf(sm.H2[s * kLdH + h], sm.w3[h], a);
#pragma unroll
        for (int o = 16; o; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        const float r = a + b3 - t[s0 + s];
        if (lane == 0) sm.dy[s] = 2.0f * r / (float)N;
        lsum = fmaf(r, r, lsum);
    }
    if (lane == 0) sm.red[warp] = lsum;
    __syncthreads();
    // dw3 = h2^T dy, db3 = sum dy; then dz2 = dy w3^T * [h2 > 0] in place of h2
    for (int h = tid; h < kH; h += kGradThreads) {
        float a = 0.f;
        for (int s = 0; s < ns; ++s) a = fmaf(sm.H2[s * kLdH + h], sm.dy[s], a);
        out[kOffW3 + h] = a;
    }
    if (tid == 0) {
        float a = 0.f, l = 0.f;
        for (int s = 0; s < ns; ++s) a += sm.dy[s];
        for (int w = 0; w < kGradThreads / 32; ++w) l += sm.red[w];
        out[kOffB3] = a;
        out[RPCA_MLP_PARAMS] = l;
    }
    __syncthreads();
    for (int e = tid; e < ns * kH; e += kGradThreads) {
        const int s = e / kH, h = e % kH;
        float &z = sm.H2[s * kLdH + h];
        z = z > 0.f ? sm.dy[s] * sm.w3[h] : 0.f;
    }
    __syncthreads();
    // dW2 = h1^T dz2, db2 = column sums of dz2
    smem_mm<true, false>(kH, kH, ns, sm.H1, kLdH, sm.H2, kLdH,
                         [&](int i, int j, float v) { out[kOffW2 + i * kH + j] = v; });
    for (int h = tid; h < kH; h += kGradThreads) {
        float a = 0.f;
        for (int s = 0; s < ns; ++s) a += sm.H2[s * kLdH + h];
        out[kOffB2 + h] = a;
    }
    // dz1 = (dz2 W2^T) * [h1 > 0]; computed in registers, then written over h1
    // (each output reads only dz2 and W2; the mask comes from the element it replaces)
    {
        constexpr int kPer = kS * kH / kGradThreads;   // 32 outputs per thread
        float v[kPer];
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int idx = tid + q * kGradThreads;
            const int i = idx / kH, j = idx % kH;
            float a = 0.f;
            if (i < ns)
                for (int k = 0; k < kH; ++k) a = fmaf(sm.H2[i * kLdH + k], sm.W2[j * kLdH + k], a);
            v[q] = a;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int idx = tid + q * kGradThreads;
            const int i = idx / kH, j = idx % kH;
            float &z = sm.H1[i * kLdH + j];
            z = (i < ns && z > 0.f) ? v[q] : 0.f;
        }
    }
    __syncthreads();
    // dW1 = F^T dz1, db1 = column sums of dz1
    smem_mm<true, false>(kF, kH, ns, sm.Fs, kLdF, sm.H1, kLdH,
                         [&](int i, int j, float v) { out[kOffW1 + i * kH + j] = v; });
    for (int h = tid; h < kH; h += kGradThreads) {
        float a = 0.f;
        for (int s = 0; s < ns; ++s) a += sm.H1[s * kLdH + h];
        out[kOffB1 + h] = a;
    }
}

__global__ void mlp_grad_reduce_kernel(const float *__restrict__ part, int nparts, int64_t N,
                                       float *__restrict__ grad, float *__restrict__ loss) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e > RPCA_MLP_PARAMS) return;
    float a = 0.f;
    for (int c = 0; c < nparts; ++c) a += part[(int64_t)c * (RPCA_MLP_PARAMS + 1) + e];
    if (e < RPCA_MLP_PARAMS) grad[e] = a;
    else if (loss) *loss = a / (float)N;
}

__global__ void mlp_adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m1,
                                float *__restrict__ m2, float lr, float b1, float b2, float eps, float c1,
                                float c2) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= RPCA_MLP_PARAMS) return;
    const float ge = g[e];
    const float a = b1 * m1[e] + (1.f - b1) * ge;
    const float v = b2 * m2[e] + (1.f - b2) * ge * ge;
    m1[e] = a;
    m2[e] = v;
    p[e] -= lr * (a * c1) / (sqrtf(v * c2) + eps);
}

__global__ void leverage_kernel(const float *__restrict__ V, int64_t n, int64_t ldv, int k, float *__restrict__ t) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    float a = 0.f;
    for (int c = 0; c < k; ++c) {
        const float v = V[j * ldv + c];
        a = fmaf(v, v, a);
    }
    t[j] = logf((float)n * a / (float)k + 1e-3f);
}

}  // namespace

}  // namespace rpca

using namespace rpca;

extern "C" int rpca_mlp_pack(const float *params, void *packed, rpca_stream_t stream) {
    if (!params || !packed || (reinterpret_cast<uintptr_t>(packed) & 15u)) return RPCA_ERR_INVALID_ARG;
    mlp_pack_kernel<<<num_sms(), 256, 0, (cudaStream_t)stream>>>(params, static_cast<uint8_t *>(packed));
    RPCA_CHECK_LAUNCH();
    return RPCA_OK;
}

extern "C" size_t rpca_mlp_forward_workspace_size(void) { return sizeof(DevStatus); }

extern "C" int rpca_mlp_forward(const void *packed, const float *F, int64_t N, float *y, float *d, void *ws,
                                size_t ws_bytes, rpca_stream_t stream) {
    if (N < 0 || !packed || (reinterpret_cast<uintptr_t>(packed) & 15u)) return RPCA_ERR_INVALID_ARG;
    if (N > 0 && (!F || (!y && !d))) return RPCA_ERR_INVALID_ARG;
    if (!ws || ws_bytes < sizeof(DevStatus)) return RPCA_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    DevStatus *st = static_cast<DevStatus *>(ws);
    if (cudaMemsetAsync(st, 0, sizeof(DevStatus), s) != cudaSuccess) return RPCA_ERR_CUDA;
    if (N == 0) return RPCA_OK;
    if (cudaFuncSetAttribute(mlp_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmem) !=
        cudaSuccess)
        return RPCA_ERR_CUDA;
    const int64_t ntiles = (N + 127) / 128;
    // two CTAs per SM: 2 x 256 TMEM columns fill the SM's 512
    const int grid = (int)std::min<int64_t>(ntiles, 2LL * num_sms());
    mlp_fwd_kernel<<<grid, kFwdThreads, kFwdSmem, s>>>(static_cast<const uint8_t *>(packed), F, N, y, d, st);
    RPCA_CHECK_LAUNCH();
    return RPCA_OK;
}

extern "C" size_t rpca_mlp_grad_workspace_size(int64_t N) {
    if (N < 1) return 0;
    return (size_t)cdiv(N, (int64_t)kS) * (RPCA_MLP_PARAMS + 1) * sizeof(float);
}

extern "C" int rpca_mlp_loss_grad(const float *params, const float *F, const float *t, int64_t N, float *grad,
                                  float *loss, void *ws, size_t ws_bytes, rpca_stream_t stream) {
    if (N < 1 || !params || !F || !t || !grad) return RPCA_ERR_INVALID_ARG;
    if (!ws || ws_bytes < rpca_mlp_grad_workspace_size(N)) return RPCA_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    const int nparts = (int)cdiv(N, (int64_t)kS);
    const size_t smem = sizeof(GradSmem);
    if (cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return RPCA_ERR_CUDA;
    float *part = static_cast<float *>(ws);
    mlp_grad_kernel<<<nparts, kGradThreads, smem, s>>>(params, F, t, N, part);
    RPCA_CHECK_LAUNCH();
    mlp_grad_reduce_kernel<<<(unsigned)cdiv(RPCA_MLP_PARAMS + 1, 256), 256, 0, s>>>(part, nparts, N, grad, loss);
    RPCA_CHECK_LAUNCH();
    return RPCA_OK;
}

extern "C" int rpca_mlp_adam(float *params, const float *grad, float *m1, float *m2, int32_t step, float lr,
                             float beta1, float beta2, float eps, rpca_stream_t stream) {
    if (!params || !grad || !m1 || !m2 || step < 1 || !(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) ||
        !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
        return RPCA_ERR_INVALID_ARG;
    const double c1 = 1.0 / (1.0 - std::pow((double)beta1, step));
    const double c2 = 1.0 / (1.0 - std::pow((double)beta2, step));
    mlp_adam_kernel<<<(unsigned)cdiv(RPCA_MLP_PARAMS, 256), 256, 0, (cudaStream_t)stream>>>(
        params, grad, m1, m2, lr, beta1, beta2, eps, (float)c1, (float)c2);
    RPCA_CHECK_LAUNCH();
    return RPCA_OK;
}

extern "C" int rpca_leverage_target(const float *V, int64_t n, int64_t ldv, int32_t k, float *t,
                                    rpca_stream_t stream) {
    if (n < 0 || k < 1 || ldv < k || (n > 0 && (!V || !t))) return RPCA_ERR_INVALID_ARG;
    if (n == 0) return RPCA_OK;
    leverage_kernel<<<(unsigned)cdiv(n, (int64_t)256), 256, 0, (cudaStream_t)stream>>>(V, n, ldv, k, t);
    RPCA_CHECK_LAUNCH();
    return RPCA_OK;
}

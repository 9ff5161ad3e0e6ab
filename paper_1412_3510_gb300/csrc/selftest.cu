// A check of the bounded device-side waits the pipelined kernels rely on.
//
// Every mbarrier wait in the library's kernels gives up after a bounded number of
// clock cycles and records RPCA_ERR_TIMEOUT in the status block, so that a lost
// arrival ends the kernel with an error the host can read instead of hanging the
// GPU.  rpca_wait_selftest runs that same wait (ptx::mbar_wait) on an mbarrier
// nothing ever arrives on, with a caller-chosen short limit, and records the
// outcome exactly as the pass kernels do.  No copy or tensor-core operation is in
// flight while it waits.
#include "internal.cuh"
#include "tc_ptx.cuh"

namespace rpca {
namespace {

__global__ void __launch_bounds__(64) wait_selftest_kernel(long long limit, DevStatus *__restrict__ st,
                                                           long long *__restrict__ waited) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        ptx::mbar_init(&bar, 1);               // expects one arrival; none comes
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const long long t0 = clock64();
        const bool ok = ptx::mbar_wait(&bar, 0, &abort_flag, limit);
        *waited = clock64() - t0;
        if (!ok) {
            atomicAdd(&st->timeouts, 1);
            dev_fail(st, RPCA_ERR_TIMEOUT);
        }
    }
    __syncthreads();
}

}  // namespace
}  // namespace rpca

extern "C" int rpca_wait_selftest(int64_t limit_cycles, int64_t *waited_cycles, void *ws, size_t ws_bytes,
                                  rpca_stream_t stream) {
    if (limit_cycles < 1000 || limit_cycles > rpca::ptx::kWaitCycles || !waited_cycles) return RPCA_ERR_INVALID_ARG;
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0 || ws_bytes < 512) return RPCA_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    auto *st = reinterpret_cast<rpca::DevStatus *>(ws);
    auto *waited = reinterpret_cast<long long *>(reinterpret_cast<char *>(ws) + 256);
    if (cudaMemsetAsync(st, 0, sizeof(rpca::DevStatus), s) != cudaSuccess) return RPCA_ERR_CUDA;
    rpca::wait_selftest_kernel<<<1, 64, 0, s>>>(limit_cycles, st, waited);
    RPCA_CHECK_LAUNCH();
    long long h = 0;
    if (cudaMemcpyAsync(&h, waited, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess) return RPCA_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return RPCA_ERR_CUDA;
    *waited_cycles = h;
    return RPCA_OK;
}

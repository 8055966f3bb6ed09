// Self-test of the bounded device-side wait used by every pipelined kernel.
//
// One thread waits on an mbarrier that nothing will ever complete, with a
// short time limit; the wait gives up, records BDCT_ERR_DEVICE_TIMEOUT in a
// status word and the kernel returns normally, so the context stays usable.
// This is how the library's kernels behave when a copy they wait for never
// lands; the self-test lets a caller confirm it without faulting anything.
#include <cuda_runtime.h>

#include "bdct_internal.h"
#include "ptx.cuh"

namespace bdct {

__global__ void k_selftest_wait(unsigned int *status, unsigned long long limit_ns)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    fence_mbar_init();
    // phase 0 never completes: no thread arrives and no copy is pending
    const unsigned long long t0 = global_ns();
    bool done = false;
    while (!done) {
        done = mbar_try_wait(&bar, 0);
        if (!done && global_ns() - t0 > limit_ns) break;
    }
    if (!done) record_timeout(status);
}

}  // namespace bdct

extern "C" int bdct_selftest_wait_timeout(unsigned int limit_us)
{
    using namespace bdct;
    if (limit_us == 0 || limit_us > 2000000u) return BDCT_ERR_INVALID_ARG;
    unsigned int *status = nullptr;
    cudaError_t e = cudaMalloc(&status, sizeof(unsigned int));
    if (e != cudaSuccess) return BDCT_ERR_CUDA;
    unsigned int v = 0;
    e = cudaMemset(status, 0, sizeof(unsigned int));
    if (e == cudaSuccess) {
        k_selftest_wait<<<1, 32>>>(status, (unsigned long long)limit_us * 1000ull);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&v, status, sizeof(v), cudaMemcpyDeviceToHost);
    cudaFree(status);
    if (e != cudaSuccess) return BDCT_ERR_CUDA;
    return (int)v;
}

// Bounded-wait check: the mbarrier wait every tensor-core kernel uses, run on a barrier
// that nothing completes, so that it gives up after its limit and reports a timeout
// through the handle's error word (include/rift_ile.h, rift_ile_wait_selftest).
#include "ile_kernels.h"
#include "tc_ptx.cuh"

namespace rift {

__global__ void wait_probe_kernel(uint64_t limit_ns, int *err)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        tc::fence_mbar_init();
    }
    __syncthreads();
    // no thread arrives: phase 0 of the barrier never completes
    if (threadIdx.x == 0 && !tc::mbar_wait(&bar, 0u, limit_ns))
        atomicOr(err, kErrTimeout);
    __syncthreads();
}

cudaError_t launch_wait_probe(uint64_t limit_ns, int *err, cudaStream_t st)
{
    wait_probe_kernel<<<1, 32, 0, st>>>(limit_ns, err);
    return cudaGetLastError();
}

}  // namespace rift

// Diagnostic kernel for the bounded-wait machinery: it waits on an mbarrier
// phase that nothing ever completes, so the wait must expire after its limit
// and record kErrSelfTest in the error word.  Used by afd_selftest_wait to
// test error reporting without hanging the GPU.
#include "afd_internal.h"
#include "afd_ptx.cuh"

namespace afd {
namespace {

__global__ void selftest_wait_kernel(uint64_t limit_ns, int *err)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);  // one arrival expected; none ever comes
        fence_mbar_init();
    }
    __syncthreads();
    mbar_wait(&bar, 0u, err, kErrSelfTest, limit_ns);
}

}  // namespace

cudaError_t launch_selftest_wait(uint64_t limit_ns, int *err, cudaStream_t stream)
{
    selftest_wait_kernel<<<1, 32, 0, stream>>>(limit_ns, err);
    return cudaGetLastError();
}

}  // namespace afd

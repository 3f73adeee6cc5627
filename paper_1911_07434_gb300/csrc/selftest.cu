// selftest.cu -- exercises the failure-detection path of the tensor-core kernels
// without faulting the GPU: one warp waits, with the same bounded mbarrier wait
// those kernels use, on a barrier that nothing ever arrives on.  The wait gives
// up after the given number of SM clocks, the kernel records FM_ERR_TIMEOUT in the
// status word the host reads, and it returns normally, so the context stays usable.
#include "tc_common.cuh"

namespace fm {
namespace {

__global__ void wait_timeout_kernel(int* status, long long limit_cycles) {
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    bool ok = true;
    if (threadIdx.x == 0) ok = tc::mbar_wait_limit(&bar, 0u, &abort_flag, limit_cycles);  // never completes
    __syncthreads();
    if (threadIdx.x == 0 && !ok) set_status(status, FM_ERR_TIMEOUT);
}

}  // namespace

cudaError_t launch_wait_timeout(int* status, long long limit_cycles, cudaStream_t s) {
    count_launch();
    wait_timeout_kernel<<<1, 32, 0, s>>>(status, limit_cycles);
    return cudaGetLastError();
}

}  // namespace fm

// hostio.cu -- the outputs of an fm_run_host batch written straight into the
// caller's host buffers by one kernel, on systems where the GPU addresses host
// memory directly (one launch in place of one copy per output buffer).
#include "fm_internal.cuh"

namespace fm {
namespace {

// One CTA per entry; every output is a whole number of 4-byte words, 4-byte aligned.
__global__ void __launch_bounds__(256) scatter_kernel(const CopyEntry* __restrict__ tab, int n) {
    pdl_enter();
    const int e = blockIdx.x;
    if (e >= n) return;
    const CopyEntry c = tab[e];
    const uint32_t* __restrict__ s = reinterpret_cast<const uint32_t*>(c.src);
    uint32_t* __restrict__ d = reinterpret_cast<uint32_t*>(c.dst);
    const int64_t words = c.bytes / 4;
    for (int64_t i = threadIdx.x; i < words; i += blockDim.x) d[i] = s[i];
}

}  // namespace

cudaError_t launch_scatter(const CopyEntry* tab, int n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    count_launch();
    launch_pdl(scatter_kernel, dim3(n), dim3(256), (size_t)(0), s, tab, n);
    return cudaGetLastError();
}

}  // namespace fm

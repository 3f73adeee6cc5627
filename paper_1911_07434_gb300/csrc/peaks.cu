// peaks.cu -- peak search of Eq. 6: the K largest local maxima of P.
//
// A local maximum is i with P[i] > P[i-1] and P[i] >= P[i+1] (a missing
// neighbour at either end never blocks).  Candidates are taken in the total
// order (P descending, index ascending).  One CTA per frame: every thread
// marks the maxima of its slice in a bit mask, then K rounds of a block-wide
// argmax (warp shuffles, then one warp over the per-warp winners) extract the
// winners in order; after each round every thread only considers candidates
// that come after the winner in that order.
#include <float.h>
#include <limits.h>

#include "fm_internal.cuh"

namespace fm {
namespace {

constexpr int kThreads = 1024;  // slice length (L + 1023) / 1024 <= 64 bits of mask (L <= 65536)

__device__ __forceinline__ bool better(float v, int i, float bv, int bi) {
    return (v > bv) || (v == bv && i < bi);
}

__device__ __forceinline__ void warp_best(float& v, int& i) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, v, off);
        const int oi = __shfl_xor_sync(0xffffffffu, i, off);
        if (better(ov, oi, v, i)) {
            v = ov;
            i = oi;
        }
    }
}

__global__ void __launch_bounds__(kThreads) peaks_kernel(const FrameDesc* __restrict__ descs) {
    __shared__ float wv[32];
    __shared__ int wi[32];
    __shared__ float gv;
    __shared__ int gi;
    const FrameDesc* dp = descs + blockIdx.x;
    const int L = dp->L, K = dp->K;
    const float* __restrict__ P = dp->P;
    const int per = (L + kThreads - 1) / kThreads;
    const int i0 = threadIdx.x * per, i1 = min(L, i0 + per);
    uint64_t mask = 0;
    for (int i = i0; i < i1; ++i) {
        const float v = P[i];
        const bool lok = (i == 0) || (v > P[i - 1]);
        const bool rok = (i == L - 1) || (v >= P[i + 1]);
        if (lok && rok) mask |= (uint64_t)1 << (i - i0);
    }
    float lastv = INFINITY;
    int lasti = -1;
    int found = 0;
    for (int k = 0; k < K; ++k) {
        float bv = -INFINITY;
        int bi = INT_MAX;
        uint64_t mm = mask;
        while (mm) {
            const int b = __ffsll((long long)mm) - 1;
            mm &= mm - 1;
            const int i = i0 + b;
            const float v = P[i];
            const bool after = (v < lastv) || (v == lastv && i > lasti);
            if (after && better(v, i, bv, bi)) {
                bv = v;
                bi = i;
            }
        }
        warp_best(bv, bi);
        if ((threadIdx.x & 31) == 0) {
            wv[threadIdx.x >> 5] = bv;
            wi[threadIdx.x >> 5] = bi;
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            float v = wv[threadIdx.x];
            int i = wi[threadIdx.x];
            warp_best(v, i);
            if (threadIdx.x == 0) {
                gv = v;
                gi = i;
            }
        }
        __syncthreads();
        const float v = gv;
        const int i = gi;
        __syncthreads();
        if (i == INT_MAX) break;
        if (threadIdx.x == 0) {
            dp->peak_idx[k] = i;
            dp->peak_deg[k] = (float)(dp->theta0 + (double)i * dp->step);
        }
        lastv = v;
        lasti = i;
        ++found;
    }
    if (threadIdx.x == 0) {
        for (int k = found; k < K; ++k) {
            dp->peak_idx[k] = -1;
            dp->peak_deg[k] = NAN;
        }
        *dp->n_peaks = found;
    }
}

}  // namespace

cudaError_t launch_peaks(const FrameDesc* d, int n_frames, int max_K, cudaStream_t s) {
    (void)max_K;
    count_launch();
    peaks_kernel<<<n_frames, kThreads, 0, s>>>(d);
    return cudaGetLastError();
}

}  // namespace fm

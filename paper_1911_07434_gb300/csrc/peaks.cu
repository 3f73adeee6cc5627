// peaks.cu -- peak search of Eq. 6: the K largest local maxima of P.
//
// A local maximum is i with P[i] > P[i-1] and P[i] >= P[i+1] (a missing
// neighbour at either end never blocks).  Candidates are taken in the total
// order (P descending, index ascending).  One CTA per frame: the frame's P is
// first copied to shared memory with coalesced loads (grids of up to kSmemL
// angles; longer ones are read in place) and every thread marks the maxima of
// its slice in a bit mask.  For K <= kWarpK every warp then extracts its own K
// best in order (K rounds of warp shuffles, each round taking the best candidate
// after the previous winner), and one warp merges the 32 sorted lists: every
// element of the global top K is in its own warp's top K, so the merge is exact.
// Larger K take K rounds of a block-wide argmax instead.
#include <float.h>
#include <limits.h>

#include "fm_internal.cuh"

namespace fm {
namespace {

constexpr int kThreads = 1024;  // slice length (L + 1023) / 1024 <= 64 bits of mask (L <= 65536)
constexpr int kSmemL = 48 * 1024;  // angles staged in shared memory (192 KB)
constexpr int kWarpK = 64;         // per-warp candidate lists up to this K

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

__global__ void __launch_bounds__(kThreads) peaks_kernel(const FrameDesc* __restrict__ descs, int staged) {
    pdl_enter();
    extern __shared__ float ps[];
    __shared__ float wv[32];
    __shared__ int wi[32];
    __shared__ float gv;
    __shared__ int gi;
    const FrameDesc* dp = descs + blockIdx.x;
    const int L = dp->L, K = dp->K;
    const float* P = dp->P;
    if (staged) {  // every frame of the launch has L <= kSmemL; eight loads in flight per thread
        for (int base = threadIdx.x; base < L; base += 8 * kThreads) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = base + u * kThreads;
                v[u] = i < L ? __ldcg(dp->P + i) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = base + u * kThreads;
                if (i < L) ps[i] = v[u];
            }
        }
        __syncthreads();
        P = ps;
    }
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
    if (K <= kWarpK) {
        __shared__ float cv[32 * kWarpK];
        __shared__ int ci[32 * kWarpK];
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int k = 0; k < K; ++k) {  // this warp's k-th best after (lastv, lasti)
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
            if (lane == 0) {
                cv[warp * kWarpK + k] = bv;
                ci[warp * kWarpK + k] = bi;
            }
            if (bi == INT_MAX) break;  // the list ends here (warp-uniform)
            lastv = bv;
            lasti = bi;
        }
        __syncthreads();
        if (warp == 0) {  // merge: lane j holds the head of warp j's list
            int ptr = 0;
            float hv = cv[lane * kWarpK];
            int hi = ci[lane * kWarpK];
            for (int k = 0; k < K; ++k) {
                float v = hv;
                int i = hi;
                warp_best(v, i);
                if (i == INT_MAX) break;
                if (hi == i) {  // indices are unique: this lane's head won
                    ++ptr;
                    hv = ptr < K ? cv[lane * kWarpK + ptr] : -INFINITY;
                    hi = ptr < K ? ci[lane * kWarpK + ptr] : INT_MAX;
                }
                if (lane == 0) {
                    dp->peak_idx[k] = i;
                    dp->peak_deg[k] = (float)(dp->theta0 + (double)i * dp->step);
                }
                ++found;
            }
            if (lane == 0) {
                for (int k = found; k < K; ++k) {
                    dp->peak_idx[k] = -1;
                    dp->peak_deg[k] = NAN;
                }
                *dp->n_peaks = found;
            }
        }
        return;
    }
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

cudaError_t launch_peaks(const FrameDesc* d, int n_frames, int max_K, int max_L, cudaStream_t s) {
    (void)max_K;
    const int staged = max_L <= kSmemL ? 1 : 0;
    const size_t smem = staged ? sizeof(float) * (size_t)max_L : 0;
    if (staged) {  // the static candidate lists and this dynamic part together pass the 48 KB default
        cudaError_t e = cudaFuncSetAttribute(peaks_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    count_launch();
    launch_pdl(peaks_kernel, dim3(n_frames), dim3(kThreads), (size_t)(smem), s, d, staged);
    return cudaGetLastError();
}

}  // namespace fm

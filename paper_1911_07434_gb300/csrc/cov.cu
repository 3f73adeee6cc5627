// cov.cu -- sample covariance R = X X^H / T (Sec. II-B, Eq. 2), FP32 SIMT path.
//
// Hermitian symmetry: only tiles (ti <= tj) of the upper block triangle are
// computed; each CTA writes its tile and the conjugate-transposed mirror
// (through a shared-memory transpose so both writes are coalesced).
// Accumulation is two-level: snapshots are summed in blocks of kChunk into a
// fresh register accumulator which is then added to the running total, which
// keeps the FP32 rounding error near sqrt(kChunk) + sqrt(T / kChunk) ulps
// instead of sqrt(T).
#include <algorithm>

#include "fm_internal.cuh"

namespace fm {
namespace {

constexpr int kTile = 64;    // output tile edge (complex elements)
constexpr int kStage = 16;   // snapshots per shared-memory stage
constexpr int kChunk = 64;   // snapshots per inner accumulation block
constexpr int kThreads = 256;
constexpr int kSmemBytes = kTile * (kTile + 1) * (int)sizeof(float2);  // >= 2 stages of A and B

__device__ __forceinline__ void tile_coords(int b, int nt, int& ti, int& tj) {
    ti = 0;
    while (b >= nt - ti) {
        b -= nt - ti;
        ++ti;
    }
    tj = ti + b;
}

__global__ void __launch_bounds__(kThreads, 2) cov_fp32_kernel(const FrameDesc* __restrict__ descs) {
    pdl_enter();
    extern __shared__ float4 smem_raw[];
    float2* smem = reinterpret_cast<float2*>(smem_raw);
    float2(*As)[kStage][kTile] = reinterpret_cast<float2(*)[kStage][kTile]>(smem);
    float2(*Bs)[kStage][kTile] = reinterpret_cast<float2(*)[kStage][kTile]>(smem + 2 * kStage * kTile);

    const FrameDesc* dp = descs + blockIdx.y;
    const int M = dp->M, T = dp->T;
    const int64_t ldx = dp->ldx;
    const float2* __restrict__ X = dp->X;
    float2* __restrict__ R = dp->R;
    const int nt = (M + kTile - 1) / kTile;
    if ((int)blockIdx.x >= nt * (nt + 1) / 2) return;
    int ti, tj;
    tile_coords(blockIdx.x, nt, ti, tj);
    const int i0 = ti * kTile, j0 = tj * kTile;

    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    // global-load mapping: row lr (0..63), 4 consecutive snapshots starting at lt
    const int lr = tid >> 2, lt = (tid & 3) * 4;
    const int ga = i0 + lr, gb = j0 + lr;
    const float2* xa = X + (int64_t)min(ga, M - 1) * ldx;
    const float2* xb = X + (int64_t)min(gb, M - 1) * ldx;
    const bool va = ga < M, vb = gb < M;

    float2 acc[4][4], tmp[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            acc[r][c] = make_float2(0.f, 0.f);
            tmp[r][c] = make_float2(0.f, 0.f);
        }

    float2 pa[4], pb[4];
    auto gload = [&](int t0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int t = t0 + lt + q;
            pa[q] = (va && t < T) ? xa[t] : make_float2(0.f, 0.f);
            pb[q] = (vb && t < T) ? xb[t] : make_float2(0.f, 0.f);
        }
    };
    auto sstore = [&](int buf) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            As[buf][lt + q][lr] = pa[q];
            Bs[buf][lt + q][lr] = pb[q];
        }
    };

    const int nstages = (T + kStage - 1) / kStage;
    gload(0);
    sstore(0);
    __syncthreads();
    for (int s = 0; s < nstages; ++s) {
        const int buf = s & 1;
        if (s + 1 < nstages) gload((s + 1) * kStage);
#pragma unroll
        for (int k = 0; k < kStage; ++k) {
            float2 a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = As[buf][k][ty + 16 * r];
#pragma unroll
            for (int c = 0; c < 4; ++c) b[c] = Bs[buf][k][tx + 16 * c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) cfmaconj(tmp[r][c], a[r], b[c]);
        }
        if (((s + 1) * kStage) % kChunk == 0 || s + 1 == nstages) {
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    acc[r][c] = cadd(acc[r][c], tmp[r][c]);
                    tmp[r][c] = make_float2(0.f, 0.f);
                }
        }
        if (s + 1 < nstages) sstore(buf ^ 1);
        __syncthreads();
    }

    const float invT = (float)(1.0 / (double)T);
    // direct tile (upper part incl. diagonal)
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int i = i0 + ty + 16 * r, j = j0 + tx + 16 * c;
            if (i < M && j < M && i <= j) {
                float2 v = cscale(acc[r][c], invT);
                if (i == j) v.y = 0.f;
                R[(int64_t)i * M + j] = v;
            }
        }
    // mirror (strictly lower part) via a padded shared-memory transpose
    float2* St = smem;  // [kTile][kTile + 1]
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) St[(ty + 16 * r) * (kTile + 1) + tx + 16 * c] = acc[r][c];
    __syncthreads();
    for (int e = tid; e < kTile * kTile; e += kThreads) {
        const int jj = e / kTile, ii = e % kTile;
        const int i = i0 + ii, j = j0 + jj;
        if (i < M && j < M && i < j) R[(int64_t)j * M + i] = cconj(cscale(St[ii * (kTile + 1) + jj], invT));
    }
}

// Copy the caller's X (leading dimension ldx_in, odd or misaligned for TMA) into
// the workspace copy the tensor-core covariance reads (even ldx, 256-byte base).
// Consecutive threads take consecutive snapshots of a row: coalesced both ways.
__global__ void repack_kernel(const FrameDesc* __restrict__ descs) {
    pdl_enter();
    const FrameDesc* dp = descs + blockIdx.y;
    if (!dp->Xin) return;
    const int M = dp->M, T = dp->T;
    const int64_t n = (int64_t)M * T;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = e / T, t = e % T;
        const_cast<float2*>(dp->X)[m * dp->ldx + t] = dp->Xin[m * dp->ldx_in + t];
    }
}

}  // namespace

cudaError_t launch_repack(const FrameDesc* d, int n_frames, int max_M, int max_T, cudaStream_t s) {
    const int64_t n = (int64_t)max_M * max_T;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 256);
    count_launch();
    launch_pdl(repack_kernel, dim3(dim3(blocks, n_frames)), dim3(256), (size_t)(0), s, d);
    return cudaGetLastError();
}

cudaError_t launch_covariance(const FrameDesc* d, int n_frames, int max_M, cudaStream_t s) {
    const int nt = (max_M + kTile - 1) / kTile;
    dim3 grid(nt * (nt + 1) / 2, n_frames);
    count_launch();
    launch_pdl(cov_fp32_kernel, dim3(grid), dim3(kThreads), (size_t)(kSmemBytes), s, d);
    return cudaGetLastError();
}

}  // namespace fm

// refine.cu -- one extra power step taken in FP32 straight from the snapshots:
//   Y = X^H V  (T x l),   C = X Y / T = R V  (M x l),
// with V = orth(C) of the preceding sketch (the power iteration of Eq. 11 /
// Alg. 2, applied once more).  When the covariance and sketch ran with TF32 or
// BF16 operands, this step hands the final Rayleigh-Ritz solve an FP32 image of
// R on the sketched subspace; it reads X twice and never forms R, so it costs
// 16 M T l real flops per frame instead of the covariance's 4 M^2 T.
//
// Both products are one batched kernel: out(a, j) = sum_k A(a, k) B(k, j) with
//   XH = true : a = snapshot t, k = antenna m, A = conj(X[m][t]), B = V, out = Y;
//   XH = false: a = antenna m,  k = snapshot t, A = X[m][t],       B = Y, out = C / T.
// A CTA owns 64 rows a and all l <= 48 columns; k runs in chunks of 32 through
// shared memory, and each thread accumulates a 4 x 3 register tile.
#include "fm_internal.cuh"

namespace fm {
namespace {

constexpr int kRows = 64, kChunk = 32, kCols = 48, kThreads = 256;

template <bool XH>
__global__ void __launch_bounds__(kThreads) xgemm_kernel(const FrameDesc* __restrict__ descs) {
    __shared__ float2 As[kChunk][kRows + 1];
    __shared__ float2 Bs[kChunk][kCols];
    const FrameDesc* dp = descs + blockIdx.y;
    if (!dp->refine) return;
    const int M = dp->M, T = dp->T, l = dp->l;
    const int n_rows = XH ? T : M, inner = XH ? M : T;
    const int a0 = blockIdx.x * kRows;
    if (a0 >= n_rows) return;
    const float2* __restrict__ X = dp->X;
    const int64_t ldx = dp->ldx;
    const float2* __restrict__ B = XH ? dp->V : dp->Y;
    const int ta = threadIdx.x % 16, tj = threadIdx.x / 16;  // rows ta + 16 r, columns 3 tj .. +2
    float2 acc[4][3];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[r][c] = make_float2(0.f, 0.f);

    for (int k0 = 0; k0 < inner; k0 += kChunk) {
        for (int e = threadIdx.x; e < kChunk * kRows; e += kThreads) {
            float2 v = make_float2(0.f, 0.f);
            if (XH) {  // consecutive threads: consecutive snapshots of one antenna row
                const int kk = e / kRows, aa = e % kRows;
                if (k0 + kk < inner && a0 + aa < n_rows) {
                    v = X[(int64_t)(k0 + kk) * ldx + a0 + aa];
                    v.y = -v.y;
                }
                As[kk][aa] = v;
            } else {   // consecutive threads: consecutive snapshots of one antenna row
                const int aa = e / kChunk, kk = e % kChunk;
                if (k0 + kk < inner && a0 + aa < n_rows) v = X[(int64_t)(a0 + aa) * ldx + k0 + kk];
                As[kk][aa] = v;
            }
        }
        for (int e = threadIdx.x; e < kChunk * kCols; e += kThreads) {
            const int kk = e / kCols, j = e % kCols;
            Bs[kk][j] = (k0 + kk < inner && j < l) ? B[(int64_t)(k0 + kk) * l + j] : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < kChunk; ++kk) {
            float2 a[4], b[3];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = As[kk][ta + 16 * r];
#pragma unroll
            for (int c = 0; c < 3; ++c) b[c] = Bs[kk][3 * tj + c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) cfma(acc[r][c], a[r], b[c]);
        }
        __syncthreads();
    }
    float2* __restrict__ out = XH ? dp->Y : dp->C;
    const float scale = XH ? 1.0f : (float)(1.0 / (double)T);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int a = a0 + ta + 16 * r;
        if (a >= n_rows) continue;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int j = 3 * tj + c;
            if (j < l) out[(int64_t)a * l + j] = make_float2(acc[r][c].x * scale, acc[r][c].y * scale);
        }
    }
}

}  // namespace

cudaError_t launch_refine(const FrameDesc* d, int n_frames, int max_M, int max_T, cudaStream_t s) {
    dim3 g1((max_T + kRows - 1) / kRows, n_frames);
    count_launch();
    xgemm_kernel<true><<<g1, kThreads, 0, s>>>(d);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dim3 g2((max_M + kRows - 1) / kRows, n_frames);
    count_launch();
    xgemm_kernel<false><<<g2, kThreads, 0, s>>>(d);
    return cudaGetLastError();
}

}  // namespace fm

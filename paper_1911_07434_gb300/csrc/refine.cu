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
// double-buffered shared memory (cp.async: the next chunk streams in while the
// current one is used), and each thread accumulates a 4 x 3 register tile.
#include "fm_internal.cuh"

namespace fm {
namespace {

constexpr int kRows = 64, kChunk = 32, kCols = 48, kThreads = 256;
constexpr int kAStride = kRows + 1;                                        // As[kk][aa] row stride
constexpr int kBufElems = kChunk * kAStride + kChunk * kCols;              // one stage, float2 units
constexpr size_t kSmemBytes = 2 * sizeof(float2) * (size_t)kBufElems;      // double-buffered

// 8-byte global -> shared copy that completes asynchronously; src_bytes = 0 fills zeros.
__device__ __forceinline__ void cp_async8(float2* dst, const float2* src, bool valid) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(valid ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Stage k-chunk k0 of A (As[kk][aa]) and B (Bs[kk][j]) into one buffer.
template <bool XH>
__device__ __forceinline__ void load_chunk(float2* buf, const float2* __restrict__ X, int64_t ldx,
                                           const float2* __restrict__ B, int l, int a0, int n_rows, int inner,
                                           int k0) {
    float2* As = buf;
    float2* Bs = buf + kChunk * kAStride;
    for (int e = threadIdx.x; e < kChunk * kRows; e += kThreads) {
        int kk, aa;
        if (XH) {  // consecutive threads: consecutive snapshots t = a of one antenna row m = k
            kk = e / kRows;
            aa = e % kRows;
        } else {   // consecutive threads: consecutive snapshots t = k of one antenna row m = a
            aa = e / kChunk;
            kk = e % kChunk;
        }
        const bool ok = (k0 + kk < inner) && (a0 + aa < n_rows);
        const int64_t off = XH ? (int64_t)(k0 + kk) * ldx + a0 + aa : (int64_t)(a0 + aa) * ldx + k0 + kk;
        cp_async8(As + kk * kAStride + aa, ok ? X + off : X, ok);
    }
    for (int e = threadIdx.x; e < kChunk * kCols; e += kThreads) {
        const int kk = e / kCols, j = e % kCols;
        const bool ok = (k0 + kk < inner) && (j < l);
        cp_async8(Bs + kk * kCols + j, ok ? B + (int64_t)(k0 + kk) * l + j : B, ok);
    }
}

template <bool XH>
__global__ void __launch_bounds__(kThreads) xgemm_kernel(const FrameDesc* __restrict__ descs) {
    pdl_enter();
    extern __shared__ float2 smem[];
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

    const int nchunks = (inner + kChunk - 1) / kChunk;
    load_chunk<XH>(smem, X, ldx, B, l, a0, n_rows, inner, 0);
    cp_async_commit();
    for (int c = 0; c < nchunks; ++c) {
        if (c + 1 < nchunks) {  // the next chunk streams in while this one is used
            load_chunk<XH>(smem + ((c + 1) & 1) * kBufElems, X, ldx, B, l, a0, n_rows, inner, (c + 1) * kChunk);
            cp_async_commit();
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const float2* As = smem + (c & 1) * kBufElems;
        const float2* Bs = As + kChunk * kAStride;
#pragma unroll 4
        for (int kk = 0; kk < kChunk; ++kk) {
            float2 a[4], b[3];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = As[kk * kAStride + ta + 16 * r];
#pragma unroll
            for (int q = 0; q < 3; ++q) b[q] = Bs[kk * kCols + 3 * tj + q];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    if (XH)
                        cfmac(acc[r][q], a[r], b[q]);  // conj(X) V
                    else
                        cfma(acc[r][q], a[r], b[q]);
                }
        }
        __syncthreads();  // the buffer is refilled two chunks later
    }
    float2* __restrict__ out = XH ? dp->Y : dp->C;
    const float scale = XH ? 1.0f : (float)(1.0 / (double)T);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int a = a0 + ta + 16 * r;
        if (a >= n_rows) continue;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const int j = 3 * tj + q;
            if (j < l) out[(int64_t)a * l + j] = make_float2(acc[r][q].x * scale, acc[r][q].y * scale);
        }
    }
}

}  // namespace

cudaError_t launch_refine(const FrameDesc* d, int n_frames, int max_M, int max_T, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(xgemm_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(xgemm_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    dim3 g1((max_T + kRows - 1) / kRows, n_frames);
    count_launch();
    launch_pdl(xgemm_kernel<true>, dim3(g1), dim3(kThreads), (size_t)(kSmemBytes), s, d);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dim3 g2((max_M + kRows - 1) / kRows, n_frames);
    count_launch();
    launch_pdl(xgemm_kernel<false>, dim3(g2), dim3(kThreads), (size_t)(kSmemBytes), s, d);
    return cudaGetLastError();
}

}  // namespace fm

// sketch.cu -- the range sketch C = R Pi of Algorithms 1 and 2 and the power
// step C = R V of Eq. 11 (Sec. III).
//
//   pass 0, projection : C = R Omega, Omega (M x l complex Gaussian) generated
//                        from Philox into shared memory, never stored.
//   pass 0, sampling   : C = R(:, I) = conj(R(I, :))^T (R is exactly Hermitian
//                        as written by the covariance kernel), I the sorted
//                        Fisher-Yates index set; rows of R are read coalesced.
//   pass p >= 1        : C = R V with V the basis from the previous orth step.
//
// The dense form is HBM-bound (R is read once per pass: 8 M^2 bytes for
// 8 M^2 l flops); each CTA owns 64 rows of R and all l columns of C.
#include "fm_internal.cuh"

namespace fm {
namespace {

constexpr int kRows = 64;     // rows of R per CTA
constexpr int kKc = 64;       // reduction chunk (columns of R / rows of Pi)
constexpr int kThreads = 256;
constexpr int kColGroups = kThreads / kRows;  // 4 threads share a row
constexpr int kMaxQ = kLMax / kColGroups;     // accumulators per thread

// dynamic smem: As[kRows][kKc+1] + Bs[kKc][l]
__global__ void __launch_bounds__(kThreads) sketch_dense_kernel(const FrameDesc* __restrict__ descs, int pass) {
    extern __shared__ float4 smem_raw[];
    float2* As = reinterpret_cast<float2*>(smem_raw);
    const FrameDesc* dp = descs + blockIdx.y;
    const int M = dp->M, l = dp->l;
    if (pass > dp->t) return;
    if (pass == 0 && dp->method != FM_RAND_PROJECTION) return;
    const int r0 = blockIdx.x * kRows;
    if (r0 >= M) return;
    float2* Bs = As + kRows * (kKc + 1);
    const float2* __restrict__ R = dp->R;
    const float2* __restrict__ V = dp->V;
    float2* __restrict__ C = dp->C;
    const uint64_t seed = dp->seed, fid = dp->frame_id;

    const int tid = threadIdx.x;
    const int row = tid / kColGroups, cg = tid % kColGroups;
    const int nq = (l - cg + kColGroups - 1) / kColGroups;  // columns cg, cg+4, ...

    float2 acc[kMaxQ], tmp[kMaxQ];
#pragma unroll
    for (int q = 0; q < kMaxQ; ++q) {
        acc[q] = make_float2(0.f, 0.f);
        tmp[q] = make_float2(0.f, 0.f);
    }

    for (int k0 = 0; k0 < M; k0 += kKc) {
        // A chunk: rows r0.., cols k0.. of R (coalesced: 64 consecutive complex per row)
        for (int e = tid; e < kRows * kKc; e += kThreads) {
            const int rr = e / kKc, kk = e % kKc;
            const int gr = r0 + rr, gk = k0 + kk;
            As[rr * (kKc + 1) + kk] = (gr < M && gk < M) ? R[(int64_t)gr * M + gk] : make_float2(0.f, 0.f);
        }
        // B chunk: rows k0.. of Omega (generated) or V
        for (int e = tid; e < kKc * l; e += kThreads) {
            const int kk = e / l, j = e % l;
            const int gk = k0 + kk;
            float2 v = make_float2(0.f, 0.f);
            if (gk < M) v = (pass == 0) ? gaussian_entry(seed, fid, gk, j) : V[(int64_t)gk * l + j];
            Bs[kk * l + j] = v;
        }
        __syncthreads();
        const float2* arow = As + row * (kKc + 1);
#pragma unroll 4
        for (int kk = 0; kk < kKc; ++kk) {
            const float2 a = arow[kk];
            const float2* brow = Bs + kk * l + cg;
#pragma unroll
            for (int q = 0; q < kMaxQ; ++q)
                if (q < nq) cfma(tmp[q], a, brow[q * kColGroups]);
        }
#pragma unroll
        for (int q = 0; q < kMaxQ; ++q) {
            acc[q] = cadd(acc[q], tmp[q]);
            tmp[q] = make_float2(0.f, 0.f);
        }
        __syncthreads();
    }
    const int gr = r0 + row;
    if (gr < M) {
#pragma unroll
        for (int q = 0; q < kMaxQ; ++q)
            if (q < nq) C[(int64_t)gr * l + cg + q * kColGroups] = acc[q];
    }
}

// pass 0, sampling: C[i][j] = conj(R[I[j]][i])
__global__ void __launch_bounds__(256) sketch_gather_kernel(const FrameDesc* __restrict__ descs) {
    extern __shared__ int ismem[];
    const FrameDesc* dp = descs + blockIdx.y;
    if (dp->method != FM_RAND_SAMPLING) return;
    const int M = dp->M, l = dp->l;
    const int i0 = blockIdx.x * 256;
    if (i0 >= M) return;
    int* perm = ismem;      // M
    int* sel = ismem + M;   // l
    if (threadIdx.x == 0) {
        sample_indices_serial(dp->seed, dp->frame_id, M, l, perm, sel);
        if (blockIdx.x == 0)
            for (int j = 0; j < l; ++j) dp->idx[j] = sel[j];
    }
    __syncthreads();
    const int i = i0 + threadIdx.x;
    if (i >= M) return;
    const float2* __restrict__ R = dp->R;
    float2* __restrict__ C = dp->C;
    for (int j = 0; j < l; ++j) C[(int64_t)i * l + j] = cconj(R[(int64_t)sel[j] * M + i]);
}

// standalone Omega / index-set generators (parity tests)
__global__ void test_matrix_kernel(uint64_t seed, uint64_t fid, int M, int l, float2* out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)M * l) return;
    out[e] = gaussian_entry(seed, fid, (int)(e / l), (int)(e % l));
}
__global__ void sample_indices_kernel(uint64_t seed, uint64_t fid, int M, int l, int* out) {
    extern __shared__ int ismem[];
    if (threadIdx.x == 0) {
        sample_indices_serial(seed, fid, M, l, ismem, ismem + M);
        for (int j = 0; j < l; ++j) out[j] = ismem[M + j];
    }
}

}  // namespace

cudaError_t launch_sketch(const FrameDesc* d, int n_frames, int max_M, int max_l, int pass, bool any_gather,
                          bool any_dense, cudaStream_t s) {
    if (pass == 0 && any_gather) {
        const size_t gsm = sizeof(int) * (size_t)(max_M + max_l);
        sketch_gather_kernel<<<dim3((max_M + 255) / 256, n_frames), 256, gsm, s>>>(d);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (!any_dense) return cudaSuccess;
    const size_t smem = sizeof(float2) * ((size_t)kRows * (kKc + 1) + (size_t)kKc * max_l);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(sketch_dense_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    sketch_dense_kernel<<<dim3((max_M + kRows - 1) / kRows, n_frames), kThreads, smem, s>>>(d, pass);
    return cudaGetLastError();
}

cudaError_t launch_test_matrix(uint64_t seed, uint64_t frame_id, int M, int l, float2* out, cudaStream_t s) {
    const int64_t n = (int64_t)M * l;
    test_matrix_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(seed, frame_id, M, l, out);
    return cudaGetLastError();
}

cudaError_t launch_sample_indices(uint64_t seed, uint64_t frame_id, int M, int l, int* out, cudaStream_t s) {
    sample_indices_kernel<<<1, 32, sizeof(int) * (size_t)(M + l), s>>>(seed, frame_id, M, l, out);
    return cudaGetLastError();
}

}  // namespace fm

// sketch.cu -- the range sketch C = R Pi of Algorithms 1 and 2 and the power
// step C = R V of Eq. 11 (Sec. III).
//
//   pass 0, projection : Omega (M x l complex Gaussian, Philox) is generated once
//                        per frame into the basis buffer V, then C = R V.
//   pass 0, sampling   : C = R(:, I) = conj(R(I, :))^T (R is exactly Hermitian
//                        as written by the covariance kernel), I the sorted
//                        Fisher-Yates index set; rows of R are read coalesced.
//   pass p >= 1        : C = R V with V the basis from the previous orth step.
//
// Dense form (the CUDA-core product, for frames the tensor-core sketch of
// sketch_tc.cu cannot read, i.e. odd M, and for fm_set_sketch_path(FM_COV_SIMT)):
// each CTA owns 64 rows of R and all l columns of C.  Threads hold a 4-row x
// ceil(l/8)-column register tile; R and V stream through double-buffered shared
// memory in 32-column chunks (cp.async: the next chunk arrives while the current
// one is consumed).  FP32 products, two-level accumulation (per chunk, then into
// the running sum).  R is read from HBM exactly once per pass.  Omega and the
// sampling gather run here for every frame.
#include "fm_internal.cuh"

namespace fm {
namespace {

constexpr int kRows = 64;      // rows of R per CTA
constexpr int kKc = 32;        // reduction chunk
constexpr int kThreads = 128;  // 16 row groups x 8 column groups
constexpr int kRowT = 4;       // rows per thread (rg + 16 r)
constexpr int kColG = 8;       // column groups (cg + 8 q)
constexpr int kMaxQ = kLMax / kColG;
constexpr int kALoads = kRows * kKc / kThreads;  // 16 complex per thread per chunk

__device__ __forceinline__ void cp_async8(void* dst, const void* src, bool valid) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(valid ? 8 : 0) : "memory");
}

template <int NQ>
__global__ void __launch_bounds__(kThreads) sketch_dense_kernel(const FrameDesc* __restrict__ descs, int pass) {
    pdl_enter();
    extern __shared__ float4 smem_raw[];
    float2(*As)[kRows][kKc + 1] = reinterpret_cast<float2(*)[kRows][kKc + 1]>(smem_raw);
    float2* Bbase = reinterpret_cast<float2*>(smem_raw) + 2 * kRows * (kKc + 1);
    const FrameDesc* dp = descs + blockIdx.y;
    const int M = dp->M, l = dp->l;
    if (pass > dp->t) return;
    if (pass == 0 && dp->method != FM_RAND_PROJECTION) return;
    if (dp->sketch_tc && sketch_on_tc(dp->method, pass)) return;  // sketch_tc.cu takes it
    const int r0 = blockIdx.x * kRows;
    if (r0 >= M) return;
    const float2* __restrict__ R = dp->R;
    const float2* __restrict__ V = dp->V;
    float2* __restrict__ C = dp->C;

    const int tid = threadIdx.x;
    const int rg = tid >> 3, cg = tid & 7;

    float2 acc[kRowT][NQ], tmp[kRowT][NQ];
#pragma unroll
    for (int r = 0; r < kRowT; ++r)
#pragma unroll
        for (int q = 0; q < NQ; ++q) acc[r][q] = tmp[r][q] = make_float2(0.f, 0.f);

    // chunk k0 of R rows (64 x 32) and of V (32 x l) into buffer buf, asynchronously
    const int nb = kKc * l;
    auto load_chunk = [&](int buf, int k0) {
#pragma unroll
        for (int u = 0; u < kALoads; ++u) {
            const int e = tid + u * kThreads;
            const int rr = e >> 5, kk = e & 31;  // kKc == 32: a warp reads 32 consecutive entries of a row
            const int gr = r0 + rr, gk = k0 + kk;
            const bool ok = gr < M && gk < M;
            cp_async8(&As[buf][rr][kk], ok ? R + (int64_t)gr * M + gk : R, ok);
        }
        for (int e = tid; e < nb; e += kThreads) {
            const int kk = e / l;
            const bool ok = k0 + kk < M;
            cp_async8(Bbase + buf * nb + e, ok ? V + (int64_t)k0 * l + e : V, ok);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };

    const int nchunks = (M + kKc - 1) / kKc;
    load_chunk(0, 0);
    for (int c = 0; c < nchunks; ++c) {
        const int buf = c & 1;
        if (c + 1 < nchunks) {  // the next chunk streams in while this one is used
            load_chunk(buf ^ 1, (c + 1) * kKc);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < kKc; ++kk) {
            float2 a[kRowT], b[NQ];
#pragma unroll
            for (int r = 0; r < kRowT; ++r) a[r] = As[buf][rg + 16 * r][kk];
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const int j = cg + kColG * q;
                b[q] = (j < l) ? Bbase[buf * nb + kk * l + j] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int r = 0; r < kRowT; ++r)
#pragma unroll
                for (int q = 0; q < NQ; ++q) cfma(tmp[r][q], a[r], b[q]);
        }
        if ((c & 3) == 3 || c + 1 == nchunks) {
#pragma unroll
            for (int r = 0; r < kRowT; ++r)
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    acc[r][q] = cadd(acc[r][q], tmp[r][q]);
                    tmp[r][q] = make_float2(0.f, 0.f);
                }
        }
        __syncthreads();  // the buffer is refilled by the next iteration's load
    }
#pragma unroll
    for (int r = 0; r < kRowT; ++r) {
        const int gr = r0 + rg + 16 * r;
        if (gr >= M) continue;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int j = cg + kColG * q;
            if (j < l) C[(int64_t)gr * l + j] = acc[r][q];
        }
    }
}

// Omega -> V for projection frames (pass 0), one thread per entry.  Frames whose first
// product runs on the tensor cores get Omega from the B-row preparation instead.
__global__ void omega_kernel(const FrameDesc* __restrict__ descs) {
    pdl_enter();
    const FrameDesc* dp = descs + blockIdx.y;
    if (dp->method != FM_RAND_PROJECTION || dp->sketch_tc) return;
    const int M = dp->M, l = dp->l;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= M * l) return;
    dp->V[e] = gaussian_entry(dp->seed, dp->frame_id, e / l, e % l);
}

// pass 0, sampling: C[i][j] = conj(R[I[j]][i])
__global__ void __launch_bounds__(256) sketch_gather_kernel(const FrameDesc* __restrict__ descs) {
    pdl_enter();
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

template <int NQ>
cudaError_t launch_dense(const FrameDesc* d, int n_frames, int max_M, int max_l, int pass, cudaStream_t s) {
    const size_t smem = sizeof(float2) * (2 * (size_t)kRows * (kKc + 1) + 2 * (size_t)kKc * max_l);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(sketch_dense_kernel<NQ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    count_launch();
    launch_pdl(sketch_dense_kernel<NQ>, dim3(dim3((max_M + kRows - 1) / kRows, n_frames)), dim3(kThreads), (size_t)(smem), s, d, pass);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sketch(const FrameDesc* d, int n_frames, int max_M, int max_l, int pass, bool any_gather,
                          bool any_omega, bool any_dense, cudaStream_t s) {
    if (pass == 0 && any_gather) {
        const size_t gsm = sizeof(int) * (size_t)(max_M + max_l);
        count_launch();
        launch_pdl(sketch_gather_kernel, dim3(dim3((max_M + 255) / 256, n_frames)), dim3(256), (size_t)(gsm), s, d);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (pass == 0 && any_omega) {
        count_launch();
        launch_pdl(omega_kernel, dim3(dim3((max_M * max_l + 255) / 256, n_frames)), dim3(256), (size_t)(0), s, d);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (!any_dense) return cudaSuccess;
    const int nq = (max_l + kColG - 1) / kColG;
    if (nq <= 1) return launch_dense<1>(d, n_frames, max_M, max_l, pass, s);
    if (nq <= 2) return launch_dense<2>(d, n_frames, max_M, max_l, pass, s);
    if (nq <= 3) return launch_dense<3>(d, n_frames, max_M, max_l, pass, s);
    if (nq <= 4) return launch_dense<4>(d, n_frames, max_M, max_l, pass, s);
    if (nq <= 6) return launch_dense<6>(d, n_frames, max_M, max_l, pass, s);
    return launch_dense<kMaxQ>(d, n_frames, max_M, max_l, pass, s);
}

cudaError_t launch_test_matrix(uint64_t seed, uint64_t frame_id, int M, int l, float2* out, cudaStream_t s) {
    const int64_t n = (int64_t)M * l;
    count_launch();
    test_matrix_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(seed, frame_id, M, l, out);
    return cudaGetLastError();
}

cudaError_t launch_sample_indices(uint64_t seed, uint64_t frame_id, int M, int l, int* out, cudaStream_t s) {
    count_launch();
    sample_indices_kernel<<<1, 32, sizeof(int) * (size_t)(M + l), s>>>(seed, frame_id, M, l, out);
    return cudaGetLastError();
}

}  // namespace fm

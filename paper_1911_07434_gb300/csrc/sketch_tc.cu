// sketch_tc.cu -- the sketch product C = R V (Sec. III, Alg. 1 / Alg. 2, Eq. 11) on the
// 5th-generation tensor cores with TF32 operands and FP32 accumulation.
//
// Real formulation on interleaved complex rows: a row of R is read as 2M FP32
// values [Rr_0, Ri_0, Rr_1, Ri_1, ...], and every column j of V becomes two B rows
//   [Vr_0, -Vi_0, Vr_1, -Vi_1, ...] -> Re C[., j],   [Vi_0, Vr_0, Vi_1, Vr_1, ...] -> Im C[., j],
// so one real GEMM D = R_rows B^T (K = 2M, N = 2 l_pad) gives C with no operand
// conversion: R streams from HBM by TMA straight into the 128-byte-swizzled
// K-major layout the MMA reads (the tensor core takes the TF32 part of each FP32
// value), and the B rows come from sketch_bprep_kernel (rounded to TF32).
//
// Which passes run here (sketch_on_tc): every pass of a frame in TF32 / BF16 mode,
// and in FP32 mode every pass but the last (pass 0 = R Omega when power steps
// follow, and the power steps before the last one): those products only select the
// subspace that the next power step refines, while the final solve reads the last
// product, which stays FP32 (sketch.cu).
//
// One CTA per 128 rows of R of one frame: warp 0 issues TMA loads (4-stage ring),
// warp 1 allocates TMEM and issues the MMAs (one thread), warps 2-5 run the
// epilogue.  Every mbarrier wait is bounded and records FM_ERR_TIMEOUT on expiry.
#include "tc_common.cuh"

namespace fm {
namespace {

using namespace tc;

constexpr int kRows = 128;
constexpr int kStageA = kRows * 128;   // 16 KB: 128 rows x 32 FP32 (16 complex)
constexpr int kMaxNB = 2 * kLMax;      // B rows (2 l_pad <= 96)
constexpr int kStageB = kMaxNB * 128;  // 12 KB
constexpr int kStage = kStageA + kStageB;
constexpr int kNStages = 4;
constexpr int kThreads = 192;
constexpr int kTiles = kNStages * kStage;
constexpr int kSmemBytes = kTiles + 1024 + 256;
constexpr uint32_t kTmemCols = 128;

__global__ void sketch_bprep_kernel(const FrameDesc* __restrict__ descs, int pass, int max_M) {
    const FrameDesc* dp = descs + blockIdx.y;
    if (!dp->sketch_tc || !sketch_on_tc(dp->method, dp->prec, dp->t, pass)) return;
    const int M = dp->M, l = dp->l, lp = sketch_tc_lpad(l);
    const int64_t rowlen = 2 * (int64_t)M;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;  // (j, m)
    if (e >= lp * M) return;
    const int j = e / M, m = e % M;
    float2 v = make_float2(0.f, 0.f);
    if (j < l) v = dp->V[(int64_t)m * l + j];
    float* re = dp->Bsk + (2 * (int64_t)j) * rowlen;
    float* im = re + rowlen;
    re[2 * m] = __uint_as_float(tf32_rn(v.x));
    re[2 * m + 1] = __uint_as_float(tf32_rn(-v.y));
    im[2 * m] = __uint_as_float(tf32_rn(v.y));
    im[2 * m + 1] = __uint_as_float(tf32_rn(v.x));
    (void)max_M;
}

__global__ void __launch_bounds__(kThreads, 1)
    sketch_tc_kernel(const FrameDesc* __restrict__ descs, const CUtensorMap* __restrict__ tmA,
                     const CUtensorMap* __restrict__ tmB, int pass) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + kTiles);
    uint64_t* full = bars;                  // [kNStages] TMA -> MMA
    uint64_t* empty = bars + kNStages;      // [kNStages] MMA -> TMA
    uint64_t* acc_full = bars + 2 * kNStages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kNStages + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + 2 * kNStages + 2);

    const FrameDesc* dp = descs + blockIdx.y;
    if (!dp->sketch_tc || !sketch_on_tc(dp->method, dp->prec, dp->t, pass)) return;
    const int M = dp->M, l = dp->l, lp = sketch_tc_lpad(l), nb = 2 * lp;
    const int r0 = blockIdx.x * kRows;
    if (r0 >= M) return;
    const int nstages = (2 * M + 31) / 32;
    const CUtensorMap* ta = tmA + blockIdx.y;
    const CUtensorMap* tb = tmB + blockIdx.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kNStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(acc_full, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(ta)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(tb)) : "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            const uint32_t bytes = (uint32_t)kStageA + (uint32_t)nb * 128u;
            for (int s = 0; s < nstages; ++s) {
                const int slot = s % kNStages;
                if (!mbar_wait(&empty[slot], ((uint32_t)(s / kNStages) & 1u) ^ 1u, abort_flag)) break;
                unsigned char* dst = base + slot * kStage;
                mbar_expect_tx(&full[slot], bytes);
                tma_load_2d(dst, ta, s * 32, r0, &full[slot]);
                tma_load_2d(dst + kStageA, tb, s * 32, 0, &full[slot]);
            }
            for (int s = max(0, nstages - kNStages); s < nstages; ++s)
                mbar_wait(&full[s % kNStages], (uint32_t)(s / kNStages) & 1u, abort_flag);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_tf32(128, (uint32_t)nb);
            for (int s = 0; s < nstages; ++s) {
                const int slot = s % kNStages;
                if (!mbar_wait(&full[slot], (uint32_t)(s / kNStages) & 1u, abort_flag)) break;
                tc_fence_after();
                const uint32_t a = sa(base + slot * kStage), b = a + kStageA;
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)  // 32 values per row = four K = 8 steps of 32 bytes
                    mma_tf32(tmem, desc_sw128(a + 32 * kk), desc_sw128(b + 32 * kk), idesc, (s > 0 || kk > 0) ? 1u : 0u);
                mma_commit(&empty[slot]);
            }
            mma_commit(acc_full);
            mbar_wait(acc_full, 0u, abort_flag);
        }
    } else {
        // epilogue: warps 2-5, TMEM lane quadrant warp % 4 = rows 32 q + lane
        const bool ok = __all_sync(0xffffffffu, mbar_wait(acc_full, 0u, abort_flag));
        tc_fence_after();
        if (ok) {
            const int q = warp & 3;
            const int row = 32 * q + lane;
            const int gr = r0 + row;
            const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16);
            float2* __restrict__ C = dp->C;
            for (int c0 = 0; c0 < nb; c0 += 16) {
                uint32_t v[16];
                tmem_ld16(tl + c0, v);
                tmem_wait_ld();
                if (gr >= M) continue;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int j = c0 / 2 + u;
                    if (j < l) C[(int64_t)gr * l + j] = make_float2(__uint_as_float(v[2 * u]), __uint_as_float(v[2 * u + 1]));
                }
            }
        }
        tc_fence_before();
    }
    __syncthreads();
    if (*abort_flag && threadIdx.x == 0) set_status(dp->status, FM_ERR_TIMEOUT);
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

}  // namespace

cudaError_t launch_sketch_tc(const FrameDesc* d, int n_frames, int max_M, int max_l, int pass, const void* tmA,
                             const void* tmB, cudaStream_t s) {
    const int lp = sketch_tc_lpad(max_l);
    count_launch();
    sketch_bprep_kernel<<<dim3((unsigned)((lp * max_M + 255) / 256), n_frames), 256, 0, s>>>(d, pass, max_M);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(sketch_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    count_launch();
    sketch_tc_kernel<<<dim3((unsigned)((max_M + kRows - 1) / kRows), n_frames), kThreads, kSmemBytes, s>>>(
        d, reinterpret_cast<const CUtensorMap*>(tmA), reinterpret_cast<const CUtensorMap*>(tmB), pass);
    return cudaGetLastError();
}

}  // namespace fm

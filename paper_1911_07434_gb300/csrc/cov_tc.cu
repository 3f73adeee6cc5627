// cov_tc.cu -- R = X X^H / T (Sec. II-B, Eq. 2) on the 5th-generation tensor
// cores: TMA loads of X tiles, tcgen05.mma (kind::tf32) into TMEM accumulators,
// tcgen05.ld epilogue.
//
// Real formulation.  With X = Xr + j Xi, one 128 x 128 output tile (I, J) of
// the upper block triangle is
//   Re R_IJ = (Xr_I Xr_J^T + Xi_I Xi_J^T) / T,  Im R_IJ = (Xi_I Xr_J^T - Xr_I Xi_J^T) / T.
// Two accumulators of 128 x 256 FP32 each (all 512 TMEM columns) hold
//   D_top = Xr_I [Xr_J; Xi_J]^T = [rr | ri],  D_bot = Xi_I [Xr_J; Xi_J]^T = [ir | ii].
// FP32 accuracy from TF32 tensor cores ("3xTF32"): every operand x is split into
// hi = rn_tf32(x) and lo = rn_tf32(x - hi), and each product is formed as
// hi*hi + hi*lo + lo*hi (the dropped lo*lo term is below 2^-22 |x y|).  The
// frame's precision mode selects this (FM_PREC_FP32), hi*hi alone (FM_PREC_TF32),
// or BF16 operands with one kind::f16 MMA per 16 snapshots (FM_PREC_BF16); the
// accumulator is FP32 in every mode.
//
// Warp roles (320 threads): warp 0 issues the TMA loads of the raw interleaved
// complex64 tiles (128 rows x 16 snapshots = one 128-byte swizzled box per
// operand and stage); warp 1 allocates TMEM and issues the MMAs (one thread);
// warps 2-9 (one row of A or of B each) split each raw stage into planar operand
// tiles in the 128-byte-swizzled K-major layout the MMA descriptors expect, and
// finally run the epilogue (TMEM -> registers -> R tile and its conjugate
// mirror).  Raw and
// converted stages are double-buffered and handed over with mbarriers; every
// wait is bounded and records FM_ERR_TIMEOUT in the frame status on expiry.
#include "tc_common.cuh"

namespace fm {
namespace {

using namespace tc;

constexpr int kTile = 128;                         // complex rows per tile side
constexpr int kRawBox = kTile * 32 * 4;            // 16 KB: 128 rows x 32 floats (16 complex)
constexpr int kConvA = kTile * 128;                // 16 KB: 128 rows x [hi 16 | lo 16] tf32
constexpr int kConvB = 2 * kTile * 128;            // 32 KB: 256 rows ([Xr_J; Xi_J]) x [hi | lo]
constexpr int kRawStage = 2 * kRawBox;             // A and B boxes
constexpr int kConvStage = 2 * kConvA + kConvB;    // Ar, Ai, B
constexpr int kNRaw = 2, kNConv = 2;
constexpr int kThreads = 320;  // warp 0 TMA, warp 1 MMA, warps 2-9 convert + epilogue
constexpr int kConv = kThreads - 64;
constexpr int kTiles = kNRaw * kRawStage + kNConv * kConvStage;   // 192 KB
constexpr int kSmemBytes = kTiles + 1024 + 256;                   // + 1024-B alignment slack + barriers
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kIdesc = idesc_tf32(128, 256);  // M = 128 rows of X_I, N = 256 rows of [Xr_J; Xi_J]
constexpr uint32_t kIdescBf16 = idesc_bf16(128, 256);

__device__ __forceinline__ void tile_coords(int b, int nt, int& ti, int& tj) {
    ti = 0;
    while (b >= nt - ti) {
        b -= nt - ti;
        ++ti;
    }
    tj = ti + b;
}

// Split 4 raw floats (2 complex) pairs into planar hi/lo (TF32-rounded) values.
__device__ __forceinline__ void split4(float a, float b, float c, float d, uint4& hi, uint4& lo) {
    hi.x = tf32_rn(a);
    hi.y = tf32_rn(b);
    hi.z = tf32_rn(c);
    hi.w = tf32_rn(d);
    lo.x = tf32_rn(a - __uint_as_float(hi.x));
    lo.y = tf32_rn(b - __uint_as_float(hi.y));
    lo.z = tf32_rn(c - __uint_as_float(hi.z));
    lo.w = tf32_rn(d - __uint_as_float(hi.w));
}

// Convert one 128-row raw box (interleaved complex, 16 per row) into the planar
// rows of two destination tiles (re -> dre row rr, im -> dim row ri):
// FP32 (3xTF32) [hi 16 | lo 16] TF32, TF32 [hi 16] only, BF16 16 values in the
// first 32 bytes of the row.
__device__ __forceinline__ void convert_row(const char* raw, int r, char* dre, int rr, char* dim, int ri, int prec) {
    if (prec == FM_PREC_BF16) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {  // output chunk h: complex 8h .. 8h+7
            const float4 v0 = *reinterpret_cast<const float4*>(raw + swz(r, 4 * h));
            const float4 v1 = *reinterpret_cast<const float4*>(raw + swz(r, 4 * h + 1));
            const float4 v2 = *reinterpret_cast<const float4*>(raw + swz(r, 4 * h + 2));
            const float4 v3 = *reinterpret_cast<const float4*>(raw + swz(r, 4 * h + 3));
            const uint4 re = make_uint4(bf16x2_rn(v0.x, v0.z), bf16x2_rn(v1.x, v1.z), bf16x2_rn(v2.x, v2.z),
                                        bf16x2_rn(v3.x, v3.z));
            const uint4 im = make_uint4(bf16x2_rn(v0.y, v0.w), bf16x2_rn(v1.y, v1.w), bf16x2_rn(v2.y, v2.w),
                                        bf16x2_rn(v3.y, v3.w));
            *reinterpret_cast<uint4*>(dre + swz(rr, h)) = re;
            *reinterpret_cast<uint4*>(dim + swz(ri, h)) = im;
        }
        return;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {  // output chunk q: complex 4q .. 4q+3
        const float4 v0 = *reinterpret_cast<const float4*>(raw + swz(r, 2 * q));
        const float4 v1 = *reinterpret_cast<const float4*>(raw + swz(r, 2 * q + 1));
        uint4 rh, rl, ih, il;
        split4(v0.x, v0.z, v1.x, v1.z, rh, rl);
        split4(v0.y, v0.w, v1.y, v1.w, ih, il);
        *reinterpret_cast<uint4*>(dre + swz(rr, q)) = rh;
        *reinterpret_cast<uint4*>(dim + swz(ri, q)) = ih;
        if (prec == FM_PREC_FP32) {
            *reinterpret_cast<uint4*>(dre + swz(rr, 4 + q)) = rl;
            *reinterpret_cast<uint4*>(dim + swz(ri, 4 + q)) = il;
        }
    }
}

__global__ void __launch_bounds__(kThreads, 1)
    cov_tc_kernel(const FrameDesc* __restrict__ descs, const CUtensorMap* __restrict__ tmaps) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char* raw = base;                              // kNRaw x {A, B}
    unsigned char* conv = base + kNRaw * kRawStage;         // kNConv x {Ar, Ai, B}
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + kTiles);
    uint64_t* raw_full = bars;                 // [kNRaw]
    uint64_t* raw_empty = bars + 2;            // [kNRaw]
    uint64_t* conv_full = bars + 4;            // [kNConv]
    uint64_t* conv_empty = bars + 6;           // [kNConv]
    uint64_t* acc_full = bars + 8;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 9);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + 10);

    const FrameDesc* dp = descs + blockIdx.y;
    const int M = dp->M, T = dp->T, prec = dp->prec;  // prec is uniform over the CTA
    const int nt = (M + kTile - 1) / kTile;
    if ((int)blockIdx.x >= nt * (nt + 1) / 2) return;
    int ti, tj;
    tile_coords(blockIdx.x, nt, ti, tj);
    const bool diag = (ti == tj);
    const int i0 = ti * kTile, j0 = tj * kTile;
    const int nstages = (T + 15) / 16;
    const CUtensorMap* tm = tmaps + blockIdx.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kNRaw; ++s) {
            mbar_init(&raw_full[s], 1);
            mbar_init(&raw_empty[s], kConv);
        }
        for (int s = 0; s < kNConv; ++s) {
            mbar_init(&conv_full[s], kConv);
            mbar_init(&conv_empty[s], 1);
        }
        mbar_init(acc_full, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        tmap_acquire(tm);
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
        // ------------------------------------------------------ TMA producer --
        if (lane == 0) {
            const uint32_t bytes = diag ? kRawBox : 2 * kRawBox;
            for (int s = 0; s < nstages; ++s) {
                const int slot = s % kNRaw;
                const uint32_t ph = (uint32_t)(s / kNRaw) & 1u;
                if (!mbar_wait(&raw_empty[slot], ph ^ 1u, abort_flag)) break;
                unsigned char* dst = raw + slot * kRawStage;
                mbar_expect_tx(&raw_full[slot], bytes);
                tma_load_2d(dst, tm, s * 32, i0, &raw_full[slot]);
                if (!diag) tma_load_2d(dst + kRawBox, tm, s * 32, j0, &raw_full[slot]);
            }
            // drain: the last loads must land before the CTA may exit
            for (int s = max(0, nstages - kNRaw); s < nstages; ++s)
                mbar_wait(&raw_full[s % kNRaw], (uint32_t)(s / kNRaw) & 1u, abort_flag);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------- MMA issuer --
        if (lane == 0) {
            const uint32_t d_top = tmem, d_bot = tmem + 256;
            for (int s = 0; s < nstages; ++s) {
                const int slot = s % kNConv;
                const uint32_t ph = (uint32_t)(s / kNConv) & 1u;
                if (!mbar_wait(&conv_full[slot], ph, abort_flag)) break;
                tc_fence_after();
                unsigned char* cv = conv + slot * kConvStage;
                const uint32_t ar = sa(cv), ai = sa(cv + kConvA), bb = sa(cv + 2 * kConvA);
                if (prec == FM_PREC_BF16) {  // one K = 16 step covers the stage's 16 snapshots
                    const uint32_t acc0 = s > 0 ? 1u : 0u;
                    mma_bf16(d_top, desc_sw128(ar), desc_sw128(bb), kIdescBf16, acc0);
                    mma_bf16(d_bot, desc_sw128(ai), desc_sw128(bb), kIdescBf16, acc0);
                } else {
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk) {
                        const uint32_t acc0 = (s > 0 || kk > 0) ? 1u : 0u;
                        const uint64_t b_hi = desc_sw128(bb + 32 * kk), b_lo = desc_sw128(bb + 64 + 32 * kk);
                        const uint64_t r_hi = desc_sw128(ar + 32 * kk), r_lo = desc_sw128(ar + 64 + 32 * kk);
                        const uint64_t i_hi = desc_sw128(ai + 32 * kk), i_lo = desc_sw128(ai + 64 + 32 * kk);
                        mma_tf32(d_top, r_hi, b_hi, kIdesc, acc0);
                        mma_tf32(d_bot, i_hi, b_hi, kIdesc, acc0);
                        if (prec == FM_PREC_FP32) {  // 3xTF32: + hi*lo + lo*hi
                            mma_tf32(d_top, r_hi, b_lo, kIdesc, 1u);
                            mma_tf32(d_top, r_lo, b_hi, kIdesc, 1u);
                            mma_tf32(d_bot, i_hi, b_lo, kIdesc, 1u);
                            mma_tf32(d_bot, i_lo, b_hi, kIdesc, 1u);
                        }
                    }
                }
                mma_commit(&conv_empty[slot]);  // frees the converted stage once these MMAs finish
            }
            mma_commit(acc_full);
            mbar_wait(acc_full, 0u, abort_flag);  // all MMAs retired before the epilogue / dealloc
        }
    } else {
        // ------------------------------------------- converters, then epilogue --
        const int r = threadIdx.x - 64;  // 0..255: row r of A (r < 128) or row r - 128 of B
        const bool is_b = r >= kTile;
        const int rr = r & (kTile - 1);
        for (int s = 0; s < nstages; ++s) {
            const int rs = s % kNRaw, cs = s % kNConv;
            if (!mbar_wait(&raw_full[rs], (uint32_t)(s / kNRaw) & 1u, abort_flag)) break;
            if (!mbar_wait(&conv_empty[cs], ((uint32_t)(s / kNConv) & 1u) ^ 1u, abort_flag)) break;
            const char* rawA = reinterpret_cast<const char*>(raw + rs * kRawStage);
            const char* rawB = diag ? rawA : rawA + kRawBox;
            char* cv = reinterpret_cast<char*>(conv + cs * kConvStage);
            if (!is_b)
                convert_row(rawA, rr, cv, rr, cv + kConvA, rr, prec);                         // Ar, Ai
            else
                convert_row(rawB, rr, cv + 2 * kConvA, rr, cv + 2 * kConvA, 128 + rr, prec);  // B = [Br; Bi]
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(&conv_full[cs]);
            mbar_arrive(&raw_empty[rs]);
        }
        // epilogue: rows 32 * (warp % 4) + lane of the tile (a warp reads only its TMEM
        // lane quadrant), complex columns [64 h, 64 h + 64) with h = 0 for warps 2-5
        // warp-uniform: tcgen05.ld below is .sync.aligned
        const bool ok = __all_sync(0xffffffffu, mbar_wait(acc_full, 0u, abort_flag));
        tc_fence_after();
        if (ok) {
            const int q = warp & 3;
            const int row = 32 * q + lane;
            const int gi = i0 + row;
            const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16);
            const float invT = (float)(1.0 / (double)T);
            float2* __restrict__ R = dp->R;
            const int h = (warp - 2) >> 2;
            for (int c0 = 64 * h; c0 < 64 * h + 64; c0 += 16) {
                uint32_t rr[16], ri[16], ir[16], ii[16];
                tmem_ld16(tl + c0, rr);
                tmem_ld16(tl + 128 + c0, ri);
                tmem_ld16(tl + 256 + c0, ir);
                tmem_ld16(tl + 384 + c0, ii);
                tmem_wait_ld();
                if (gi >= M) continue;
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    const int gj = j0 + c0 + c;
                    if (gj >= M || (diag && gj < gi)) continue;
                    float re = (__uint_as_float(rr[c]) + __uint_as_float(ii[c])) * invT;
                    float im = (__uint_as_float(ir[c]) - __uint_as_float(ri[c])) * invT;
                    if (gj == gi) im = 0.f;
                    R[(int64_t)gi * M + gj] = make_float2(re, im);
                    if (gj != gi) R[(int64_t)gj * M + gi] = make_float2(re, -im);
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

size_t cov_tc_smem_bytes() { return kSmemBytes; }

cudaError_t launch_covariance_tc(const FrameDesc* d, const void* tmaps, int n_frames, int max_M, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(cov_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    const int nt = (max_M + kTile - 1) / kTile;
    dim3 grid(nt * (nt + 1) / 2, n_frames);
    count_launch();
    cov_tc_kernel<<<grid, kThreads, kSmemBytes, s>>>(d, reinterpret_cast<const CUtensorMap*>(tmaps));
    return cudaGetLastError();
}

}  // namespace fm

// scan_tc.cu -- MUSIC pseudo-spectrum (Eq. 5 / Eq. 10) for a batch of frames on
// the 5th-generation tensor cores.
//
// Frames that share M and the angle grid share their steering vectors, so the
// scan of a batch is one real GEMM per 128-angle tile:
//   D[i][n] = sum_k A[i][k] B[n][k],  A = steering rows [ar_0, ai_0, ar_1, ai_1, ...]
//   (a_m = ar + j ai = e^{j pi m q_i}, or e^{j pi x_m q_i} for a group whose array has
//   explicit element positions x_m), B = two rows per (frame f, column k of U_s):
//   [ur_m, ui_m]_m -> Re(u^H a),  [-ui_m, ur_m]_m -> Im(u^H a),
// and P_f(i) = 1 / (M - sum_k (Re^2 + Im^2)).  A is generated in registers by
// the CTA itself (the exact phase reduction of scan.cu, one sincospi per
// element) and written to shared memory as hi/lo pairs; B (U_s of up to
// 512 / (2 ncp) frames, already split into hi/lo by scan_bprep_kernel) arrives by
// TMA.  Each FP32 product is formed as hi*hi + hi*lo + lo*hi.  In the FP32 mode the
// pairs are FP16 (kind::f16, twice the TF32 rate): both operands are bounded a priori
// (|a_m| = 1, U_s has unit columns), so scaled by 2^8 they stay below 2^8, hi + lo
// carries 22 significant bits whenever lo is a normal FP16 value and otherwise misses
// x by at most 2^-25 (2^-33 unscaled), and the products match 3xTF32 accuracy; a stage
// is 16 antennas.  The batch's precision mode may instead take TF32 hi*hi alone
// (FM_PREC_TF32) or BF16 operands (FM_PREC_BF16, one MMA per 8 antennas); those
// stages are 8 antennas.  Two 128 x 256 FP32 accumulators fill the 512 TMEM columns.
//
// Warp roles (320 threads): warp 0 TMA producer, warp 1 TMEM allocation + MMA
// issue, warps 2-9 steering generation (two threads per angle row, half of each
// stage's antennas each) and the epilogue.
#include "tc_common.cuh"

namespace fm {
namespace {

using namespace tc;

constexpr int kRowsA = 128;                // angles per tile
constexpr int kRowsB = 512;                // rows of B per CTA (two accumulators of N = 256)
constexpr int kStageA = kRowsA * 128;      // 16 KB: [hi 16 | lo 16] floats per angle row
constexpr int kStageB = kRowsB * 128;      // 64 KB
constexpr int kStage = kStageA + kStageB;
constexpr int kNStages = 2;
constexpr int kThreads = 320;  // warp 0 TMA, warp 1 MMA, warps 2-9 steering + epilogue
constexpr int kTiles = kNStages * kStage;  // 160 KB
constexpr int kSmemBytes = kTiles + 1024 + 256;
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kIdesc = idesc_tf32(128, 256);
constexpr uint32_t kIdescBf16 = idesc_bf16(128, 256);
constexpr uint32_t kIdescF16 = idesc_f16(128, 256);
constexpr float kScaleF16 = 256.f;          // both FP16 operands of the FP32 mode
constexpr float kUnscaleF16 = 1.f / 65536.f;  // exact: 2^-16 on the accumulator

// antennas per stage: 16 in the FP32 mode (two K = 16 FP16 steps), 8 otherwise
__host__ __device__ inline int scan_stage_ant(int prec) { return prec == FM_PREC_FP32 ? 16 : 8; }

__device__ __forceinline__ void split2(float a, float b, uint32_t* hi, uint32_t* lo) {
    hi[0] = tf32_rn(a);
    hi[1] = tf32_rn(b);
    lo[0] = tf32_rn(a - __uint_as_float(hi[0]));
    lo[1] = tf32_rn(b - __uint_as_float(hi[1]));
}

// B rows for the frames of one launch: row f*2ncp + 2k (Re) and + 1 (Im).  TF32 and
// BF16 modes: along a row, stage s (8 antennas) holds 32 floats [hi of 16 interleaved
// values | lo] (BF16: 16 values in the first 32 bytes).  FP32 mode: stage s (16
// antennas, 128 bytes) holds FP16 [hi | lo] of the values of antennas 16s .. 16s+7,
// then [hi | lo] of antennas 16s+8 .. 16s+15, scaled by 2^8 (the first half of the row).
__global__ void scan_bprep_kernel(const FrameDesc* __restrict__ descs, int n_frames, int M, int Mp, int ncp, int prec,
                                  float* __restrict__ Bp) {
    pdl_enter();
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // (f, k, m)
    const int64_t total = (int64_t)n_frames * ncp * Mp;
    if (e >= total) return;
    const int m = (int)(e % Mp);
    const int k = (int)((e / Mp) % ncp);
    const int f = (int)(e / ((int64_t)Mp * ncp));
    const FrameDesc* dp = descs + f;
    float2 u = make_float2(0.f, 0.f);
    if (m < M && k < dp->ncols) u = dp->Us[(int64_t)m * dp->kpad + k];
    const int64_t rowlen = 4 * (int64_t)Mp;
    float* re_row = Bp + ((int64_t)f * 2 * ncp + 2 * k) * rowlen;
    float* im_row = re_row + rowlen;
    if (prec == FM_PREC_FP32) {
        uint32_t* re_w = reinterpret_cast<uint32_t*>(re_row);
        uint32_t* im_w = reinterpret_cast<uint32_t*>(im_row);
        const int at = (m >> 4) * 32 + ((m >> 3) & 1) * 16 + (m & 7);  // 4-byte words
        uint32_t hi, lo;
        split_f16x2(kScaleF16 * u.x, kScaleF16 * u.y, hi, lo);  // Re row: [ur, ui]
        re_w[at] = hi;
        re_w[at + 8] = lo;
        split_f16x2(-kScaleF16 * u.y, kScaleF16 * u.x, hi, lo);  // Im row: [-ui, ur]
        im_w[at] = hi;
        im_w[at + 8] = lo;
        return;
    }
    const int s = m >> 3, p = (2 * m) & 15;
    if (prec == FM_PREC_BF16) {  // 16 BF16 values in the first 32 bytes of the stage's 128
        reinterpret_cast<uint32_t*>(re_row)[s * 32 + p / 2] = bf16x2_rn(u.x, u.y);
        reinterpret_cast<uint32_t*>(im_row)[s * 32 + p / 2] = bf16x2_rn(-u.y, u.x);
        return;
    }
    uint32_t hi[2], lo[2];
    split2(u.x, u.y, hi, lo);  // Re row: [ur, ui]
    re_row[s * 32 + p] = __uint_as_float(hi[0]);
    re_row[s * 32 + p + 1] = __uint_as_float(hi[1]);
    re_row[s * 32 + 16 + p] = __uint_as_float(lo[0]);
    re_row[s * 32 + 16 + p + 1] = __uint_as_float(lo[1]);
    split2(-u.y, u.x, hi, lo);  // Im row: [-ui, ur]
    im_row[s * 32 + p] = __uint_as_float(hi[0]);
    im_row[s * 32 + p + 1] = __uint_as_float(hi[1]);
    im_row[s * 32 + 16 + p] = __uint_as_float(lo[0]);
    im_row[s * 32 + 16 + p + 1] = __uint_as_float(lo[1]);
}

// Steering entry m of angle row (q_hi, q_lo): a uniform array, or the element
// positions of the scan group (POS; every frame of a group shares them).
// Angle ia of frame fo goes to the main-lobe recompute when ||U_s^H a||^2 = M - den
// exceeds 4 ncols (or den is NaN).  Warp-wide: the flagged lanes take consecutive
// entries of the frame's list (one atomic per warp); `frame_ok` and fo are uniform.
// The epilogue's per-frame outputs, copied from the descriptors to shared memory once per
// CTA (the epilogue would otherwise wait on a descriptor load for every frame it writes).
struct FrameOut {
    float* P;
    float* Pdb;
    int* fix_count;
    int* fix_list;
    float lobe;  // main-lobe threshold 4 ncols
};

__device__ __forceinline__ void list_main_lobe(const FrameOut& fo, bool frame_ok, int ia, int L, float Mf, float den,
                                               int lane) {
    const bool flag = frame_ok && ia < L && !(den >= Mf - fo.lobe);
    const unsigned bal = __ballot_sync(0xffffffffu, flag);
    if (!bal) return;
    int base = 0;
    if (lane == 0) base = atomicAdd(fo.fix_count, __popc(bal));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (flag) fo.fix_list[base + __popc(bal & ((1u << lane) - 1u))] = ia;
}

template <bool POS>
__device__ __forceinline__ float2 steer_elem(int m, float2 qq, const float2* __restrict__ pos) {
    if constexpr (POS)
        return steer_pos(pos[m], qq.x, qq.y);
    else
        return steer_exact(m, qq.x, qq.y);
}

template <int NCP, bool POS>
__global__ void __launch_bounds__(kThreads, 1)
    scan_tc_kernel(const FrameDesc* __restrict__ descs, int n_frames, const CUtensorMap* __restrict__ tmB, int M,
                   int Mp, int L, int prec) {
    pdl_enter();
    constexpr int kRowsPerFrame = 2 * NCP;
    constexpr int kFramesPerCta = kRowsB / kRowsPerFrame;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + kTiles);
    uint64_t* a_full = bars;      // [2] generators -> MMA
    uint64_t* b_full = bars + 2;  // [2] TMA -> MMA
    uint64_t* empty = bars + 4;   // [2] MMA -> TMA and generators
    uint64_t* acc_full = bars + 6;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 7);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + 8);

    const int f0 = blockIdx.y * kFramesPerCta;
    const int nf = min(kFramesPerCta, n_frames - f0);
    if (nf <= 0) return;
    const int nrows = nf * kRowsPerFrame;
    const bool two = nrows > 256;
    const int i0 = blockIdx.x * kRowsA;
    const int nstages = Mp / scan_stage_ant(prec);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kNStages; ++s) {
            mbar_init(&a_full[s], kThreads - 64);
            mbar_init(&b_full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(acc_full, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        tmap_acquire(tmB);
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    __shared__ FrameOut fout[kFramesPerCta];
    for (int f = threadIdx.x; f < nf; f += kThreads) {
        const FrameDesc* dp = descs + f0 + f;
        fout[f] = FrameOut{dp->P, dp->Pdb, dp->fix_count, dp->fix_list, 4.0f * (float)dp->ncols};
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            const uint32_t bytes = (two ? 2u : 1u) * 256u * 128u;
            const int y0 = f0 * kRowsPerFrame;
            for (int s = 0; s < nstages; ++s) {
                const int slot = s % kNStages;
                if (!mbar_wait(&empty[slot], ((uint32_t)(s / kNStages) & 1u) ^ 1u, abort_flag)) break;
                unsigned char* bdst = base + slot * kStage + kStageA;
                mbar_expect_tx(&b_full[slot], bytes);
                tma_load_2d(bdst, tmB, s * 32, y0, &b_full[slot]);
                if (two) tma_load_2d(bdst + 256 * 128, tmB, s * 32, y0 + 256, &b_full[slot]);
            }
            for (int s = max(0, nstages - kNStages); s < nstages; ++s)
                mbar_wait(&b_full[s % kNStages], (uint32_t)(s / kNStages) & 1u, abort_flag);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            for (int s = 0; s < nstages; ++s) {
                const int slot = s % kNStages;
                const uint32_t ph = (uint32_t)(s / kNStages) & 1u;
                if (!mbar_wait(&a_full[slot], ph, abort_flag)) break;
                if (!mbar_wait(&b_full[slot], ph, abort_flag)) break;
                tc_fence_after();
                const uint32_t a = sa(base + slot * kStage), b = a + kStageA;
                if (prec == FM_PREC_BF16) {  // one K = 16 step per stage
                    const uint32_t acc0 = s > 0 ? 1u : 0u;
                    mma_bf16(tmem, desc_sw128(a), desc_sw128(b), kIdescBf16, acc0);
                    if (two) mma_bf16(tmem + 256, desc_sw128(a), desc_sw128(b + 256 * 128), kIdescBf16, acc0);
                } else if (prec == FM_PREC_FP32) {  // two K = 16 FP16 steps: [hi | lo] at 64 kk
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk) {
                        const uint32_t acc0 = (s > 0 || kk > 0) ? 1u : 0u;
                        const uint64_t a_hi = desc_sw128(a + 64 * kk), a_lo = desc_sw128(a + 64 * kk + 32);
                        const uint64_t b0_hi = desc_sw128(b + 64 * kk), b0_lo = desc_sw128(b + 64 * kk + 32);
                        mma_bf16(tmem, a_hi, b0_hi, kIdescF16, acc0);
                        mma_bf16(tmem, a_hi, b0_lo, kIdescF16, 1u);
                        mma_bf16(tmem, a_lo, b0_hi, kIdescF16, 1u);
                        if (two) {
                            const uint32_t b1 = b + 256 * 128;
                            const uint64_t b1_hi = desc_sw128(b1 + 64 * kk), b1_lo = desc_sw128(b1 + 64 * kk + 32);
                            mma_bf16(tmem + 256, a_hi, b1_hi, kIdescF16, acc0);
                            mma_bf16(tmem + 256, a_hi, b1_lo, kIdescF16, 1u);
                            mma_bf16(tmem + 256, a_lo, b1_hi, kIdescF16, 1u);
                        }
                    }
                } else {
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk) {
                        const uint32_t acc0 = (s > 0 || kk > 0) ? 1u : 0u;
                        const uint64_t a_hi = desc_sw128(a + 32 * kk), a_lo = desc_sw128(a + 64 + 32 * kk);
                        const uint64_t b0_hi = desc_sw128(b + 32 * kk), b0_lo = desc_sw128(b + 64 + 32 * kk);
                        mma_tf32(tmem, a_hi, b0_hi, kIdesc, acc0);
                        if (prec == FM_PREC_FP32) {
                            mma_tf32(tmem, a_hi, b0_lo, kIdesc, 1u);
                            mma_tf32(tmem, a_lo, b0_hi, kIdesc, 1u);
                        }
                        if (two) {
                            const uint32_t b1 = b + 256 * 128;
                            const uint64_t b1_hi = desc_sw128(b1 + 32 * kk), b1_lo = desc_sw128(b1 + 64 + 32 * kk);
                            mma_tf32(tmem + 256, a_hi, b1_hi, kIdesc, acc0);
                            if (prec == FM_PREC_FP32) {
                                mma_tf32(tmem + 256, a_hi, b1_lo, kIdesc, 1u);
                                mma_tf32(tmem + 256, a_lo, b1_hi, kIdesc, 1u);
                            }
                        }
                    }
                }
                mma_commit(&empty[slot]);
            }
            mma_commit(acc_full);
            mbar_wait(acc_full, 0u, abort_flag);
        }
    } else {
        // ------------------------------------------ steering generation --------
        // two threads per angle row: half g generates antenna pairs c = 2 g, 2 g + 1 of each stage
        const int r = (threadIdx.x - 64) & (kRowsA - 1), g = (threadIdx.x - 64) >> 7;
        const int i = i0 + r;
        const float2 qq = (i < L) ? descs[0].qtab[i] : make_float2(0.f, 0.f);
        const float2* __restrict__ pos = descs[0].pos;
        // FP32 mode, uniform array: a_{m + u} = a_m a_u, so this thread's 8 antennas of a stage
        // (16 s + 8 g + u) are one exactly reduced base value times a_u (u < 8, computed once);
        // each product adds about 2u of rounding to entries accurate to about u
        float2 w8[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) w8[u] = steer_exact(u, qq.x, qq.y);
        for (int s = 0; s < nstages; ++s) {
            const int slot = s % kNStages;
            if (!mbar_wait(&empty[slot], ((uint32_t)(s / kNStages) & 1u) ^ 1u, abort_flag)) break;
            char* arow = reinterpret_cast<char*>(base + slot * kStage);
            if (prec == FM_PREC_BF16) {  // 16 BF16 values (8 antennas) in the row's first 32 bytes
#pragma unroll
                for (int cc = 0; cc < 2; ++cc) {
                    const int c = 2 * g + cc;
                    const int m0 = 8 * s + 2 * c;
                    const float2 a0 = (i < L && m0 < M) ? steer_elem<POS>(m0, qq, pos) : make_float2(0.f, 0.f);
                    const float2 a1 = (i < L && m0 + 1 < M) ? steer_elem<POS>(m0 + 1, qq, pos) : make_float2(0.f, 0.f);
                    *reinterpret_cast<uint2*>(arow + swz(r, c >> 1) + 8 * (c & 1)) =
                        make_uint2(bf16x2_rn(a0.x, a0.y), bf16x2_rn(a1.x, a1.y));
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(&a_full[slot]);
                continue;
            }
            if (prec == FM_PREC_FP32) {  // antennas 16s + 8g .. +7: FP16 hi in 16-byte chunks 4g, 4g+1, lo in 4g+2, 4g+3
#pragma unroll
                const int mb = 16 * s + 8 * g;
                const float2 ab = POS ? make_float2(0.f, 0.f) : steer_exact(mb, qq.x, qq.y);
                for (int cc = 0; cc < 2; ++cc) {
                    uint4 hi, lo;
                    uint32_t* hv = reinterpret_cast<uint32_t*>(&hi);
                    uint32_t* lv = reinterpret_cast<uint32_t*>(&lo);
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int m = mb + 4 * cc + u;
                        float2 a = make_float2(0.f, 0.f);
                        if (i < L && m < M) a = POS ? steer_elem<POS>(m, qq, pos) : cmul(ab, w8[4 * cc + u]);
                        split_f16x2(kScaleF16 * a.x, kScaleF16 * a.y, hv[u], lv[u]);
                    }
                    *reinterpret_cast<uint4*>(arow + swz(r, 4 * g + cc)) = hi;
                    *reinterpret_cast<uint4*>(arow + swz(r, 4 * g + 2 + cc)) = lo;
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(&a_full[slot]);
                continue;
            }
#pragma unroll
            for (int cc = 0; cc < 2; ++cc) {  // chunk c: antennas 8s + 2c, 8s + 2c + 1
                const int c = 2 * g + cc;
                uint4 hi, lo;
                uint32_t h[2], w[2];
                const int m0 = 8 * s + 2 * c;
                float2 a0 = (i < L && m0 < M) ? steer_elem<POS>(m0, qq, pos) : make_float2(0.f, 0.f);
                float2 a1 = (i < L && m0 + 1 < M) ? steer_elem<POS>(m0 + 1, qq, pos) : make_float2(0.f, 0.f);
                split2(a0.x, a0.y, h, w);
                hi.x = h[0];
                hi.y = h[1];
                lo.x = w[0];
                lo.y = w[1];
                split2(a1.x, a1.y, h, w);
                hi.z = h[0];
                hi.w = h[1];
                lo.z = w[0];
                lo.w = w[1];
                *reinterpret_cast<uint4*>(arow + swz(r, c)) = hi;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(&a_full[slot]);
        }
        // ---------------------------------------------------------- epilogue --
        const bool ok = __all_sync(0xffffffffu, mbar_wait(acc_full, 0u, abort_flag));
        tc_fence_after();
        if (ok) {
            // a warp reads its TMEM lane quadrant; the two warps of a quadrant split the columns
            const int q = warp & 3, half = (warp - 2) >> 2;
            const int row = 32 * q + lane;
            const int ia = i0 + row;
            const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16);
            const float Mf = (float)M;
            const float us = prec == FM_PREC_FP32 ? kUnscaleF16 : 1.f;  // exact power of two
            if constexpr (kRowsPerFrame <= 16) {
                const int nchunks = (nrows + 15) / 16;
                constexpr int kB = 4;  // TMEM loads in flight per wait
                for (int c0 = half; c0 < nchunks; c0 += 2 * kB) {
                    uint32_t vb[kB][16];
#pragma unroll
                    for (int b = 0; b < kB; ++b)
                        if (c0 + 2 * b < nchunks) tmem_ld16(tl + 16 * (c0 + 2 * b), vb[b]);
                    tmem_wait_ld();
#pragma unroll
                    for (int b = 0; b < kB; ++b) {
                    const int ch = c0 + 2 * b;
                    if (ch >= nchunks) break;
                    const uint32_t* v = vb[b];
#pragma unroll
                    for (int j = 0; j < 16; j += kRowsPerFrame) {
                        float acc = 0.f;
#pragma unroll
                        for (int jj = 0; jj < kRowsPerFrame; ++jj) {
                            const float x = __uint_as_float(v[j + jj]) * us;
                            acc = fmaf(x, x, acc);
                        }
                        const int f = (16 * ch + j) / kRowsPerFrame;
                        const float den = Mf - acc;
                        const FrameOut& fo = fout[min(f, nf - 1)];
                        if (f < nf && ia < L) {
                            const float P = (den > 0.f) ? 1.0f / den : INFINITY;
                            fo.P[ia] = P;
                            if (fo.Pdb) fo.Pdb[ia] = 10.0f * log10f(fminf(P, 3.402823466e38f));
                        }
                        list_main_lobe(fo, f < nf, ia, L, Mf, den, lane);
                    }
                    }
                }
            } else {
                for (int f = half; f < nf; f += 2) {
                    float acc = 0.f;
#pragma unroll
                    for (int h = 0; h < kRowsPerFrame / 16; ++h) {
                        uint32_t v[16];
                        tmem_ld16(tl + f * kRowsPerFrame + 16 * h, v);
                        tmem_wait_ld();
#pragma unroll
                        for (int jj = 0; jj < 16; ++jj) {
                            const float x = __uint_as_float(v[jj]) * us;
                            acc = fmaf(x, x, acc);
                        }
                    }
                    const float den = Mf - acc;
                    const FrameOut& fo = fout[f];
                    if (ia < L) {
                        const float P = (den > 0.f) ? 1.0f / den : INFINITY;
                        fo.P[ia] = P;
                        if (fo.Pdb) fo.Pdb[ia] = 10.0f * log10f(fminf(P, 3.402823466e38f));
                    }
                    list_main_lobe(fo, true, ia, L, Mf, den, lane);
                }
            }
        }
        tc_fence_before();
    }
    __syncthreads();
    if (*abort_flag && threadIdx.x == 0) {
        for (int f = 0; f < nf; ++f) set_status(descs[f0 + f].status, FM_ERR_TIMEOUT);
    }
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

template <int NCP, bool POS>
cudaError_t launch_ncp_t(const FrameDesc* d, int n_frames, const void* tmB, int M, int Mp, int L, int prec,
                         cudaStream_t s) {
    cudaError_t e =
        cudaFuncSetAttribute(scan_tc_kernel<NCP, POS>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    const int fpc = kRowsB / (2 * NCP);
    dim3 grid((L + kRowsA - 1) / kRowsA, (n_frames + fpc - 1) / fpc);
    count_launch();
    launch_pdl(scan_tc_kernel<NCP, POS>, dim3(grid), dim3(kThreads), (size_t)(kSmemBytes), s, d, n_frames, reinterpret_cast<const CUtensorMap*>(tmB),
                                                                M, Mp, L, prec);
    return cudaGetLastError();
}

template <int NCP>
cudaError_t launch_ncp(const FrameDesc* d, int n_frames, const void* tmB, int M, int Mp, int L, int prec, bool pos,
                       cudaStream_t s) {
    return pos ? launch_ncp_t<NCP, true>(d, n_frames, tmB, M, Mp, L, prec, s)
               : launch_ncp_t<NCP, false>(d, n_frames, tmB, M, Mp, L, prec, s);
}

}  // namespace

int scan_tc_ncp(int ncols) {
    int p = 1;
    while (p < ncols) p *= 2;
    return p;
}

cudaError_t launch_scan_tc(const FrameDesc* d, int n_frames, int M, int ncols, int L, int prec, bool pos, float* bprep,
                           const void* tmB, cudaStream_t s) {
    const int ncp = scan_tc_ncp(ncols);
    const int Mp = scan_tc_mp(M);
    const int64_t total = (int64_t)n_frames * ncp * Mp;
    count_launch();
    launch_pdl(scan_bprep_kernel, dim3((unsigned)((total + 255) / 256)), dim3(256), (size_t)(0), s, d, n_frames, M, Mp, ncp, prec, bprep);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    switch (ncp) {
        case 1: return launch_ncp<1>(d, n_frames, tmB, M, Mp, L, prec, pos, s);
        case 2: return launch_ncp<2>(d, n_frames, tmB, M, Mp, L, prec, pos, s);
        case 4: return launch_ncp<4>(d, n_frames, tmB, M, Mp, L, prec, pos, s);
        case 8: return launch_ncp<8>(d, n_frames, tmB, M, Mp, L, prec, pos, s);
        default: return launch_ncp<16>(d, n_frames, tmB, M, Mp, L, prec, pos, s);
    }
}

}  // namespace fm

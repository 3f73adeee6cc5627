// cov_tc.cu -- R = X X^H / T (Sec. II-B, Eq. 2) on the 5th-generation tensor
// cores: TMA loads of X tiles, tcgen05.mma (kind::tf32) into TMEM accumulators,
// tcgen05.ld epilogue staged through shared memory.
//
// Real formulation.  With X = Xr + j Xi, one 128 x 128 output tile (I, J) of
// the upper block triangle is
//   Re R_IJ = (Xr_I Xr_J^T + Xi_I Xi_J^T) / T,  Im R_IJ = (Xi_I Xr_J^T - Xr_I Xi_J^T) / T.
// An off-diagonal tile takes two accumulators of 128 x 256 FP32 (all 512 TMEM columns):
//   D_top = Xr_I [Xr_J; Xi_J]^T = [rr | ri],  D_bot = Xi_I [Xr_J; Xi_J]^T = [ir | ii].
// A diagonal tile (I = J) needs only three of the four blocks: ir = ri^T there, so
//   D_top = Xr_I [Xr_I; Xi_I]^T = [rr | ri] and D_bot = Xi_I Xi_I^T = ii (N = 128),
// and Im R_II = ri^T - ri is formed in the epilogue through shared memory; its A
// operands are the two halves of its own converted B tile, so only the B rows are
// converted.  FP32 accuracy from TF32 tensor cores ("3xTF32"): every operand x is
// split into hi = rn_tf32(x) and lo = rn_tf32(x - hi), and each product is formed as
// hi*hi + hi*lo + lo*hi (the dropped lo*lo term is below 2^-22 |x y|).  The frame's
// precision mode selects this (FM_PREC_FP32), hi*hi alone (FM_PREC_TF32), or BF16
// operands with one kind::f16 MMA per 16 snapshots (FM_PREC_BF16); the accumulator
// is FP32 in every mode.
//
// Work items.  Each CTA runs one CovItem: a tile, or a range of its 16-snapshot
// stages.  The host orders the items longest first and splits the tiles that would
// otherwise run alone in the last, partial wave along T; the parts of a split tile
// write their partial tiles to a workspace, and the part that finishes last (a
// device-scope counter, no waiting) adds them in part order -- a fixed order, so the
// result does not depend on which part finished last -- and writes R.
//
// Warp roles (320 threads): warp 0 issues the TMA loads of the raw interleaved
// complex64 tiles (128 rows x 16 snapshots = one 128-byte swizzled box per
// operand and stage); warp 1 allocates TMEM and issues the MMAs (one thread);
// warps 2-9 split each raw stage into planar operand tiles in the 128-byte-swizzled
// K-major layout the MMA descriptors expect, and finally run the epilogue (TMEM ->
// registers -> a tile in shared memory -> coalesced row stores of R and of its
// conjugate mirror).  Three raw and two converted stages are handed over with
// mbarriers; every wait is bounded and records FM_ERR_TIMEOUT in the frame status on
// expiry.
#include "tc_common.cuh"

namespace fm {
namespace {

using namespace tc;

constexpr int kTile = kCovTile;                    // complex rows per tile side
constexpr int kRawBox = kTile * 32 * 4;            // 16 KB: 128 rows x 32 floats (16 complex)
constexpr int kConvA = kTile * 128;                // 16 KB: 128 rows x [hi 16 | lo 16] tf32
constexpr int kConvB = 2 * kTile * 128;            // 32 KB: 256 rows ([Xr_J; Xi_J]) x [hi | lo]
constexpr int kRawStage = 2 * kRawBox;             // A and B boxes
constexpr int kConvStage = 2 * kConvA + kConvB;    // Ar, Ai, B
constexpr int kNRaw = 3, kNConv = 2;
constexpr int kThreads = 320;  // warp 0 TMA, warp 1 MMA, warps 2-9 convert + epilogue
constexpr int kConv = kThreads - 64;
constexpr int kTiles = kNRaw * kRawStage + kNConv * kConvStage;   // 224 KB
constexpr int kSmemBytes = kTiles + 1024 + 256;                   // + 1024-B alignment slack + barriers
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kIdesc = idesc_tf32(128, 256);  // M = 128 rows of X_I, N = 256 rows of [Xr_J; Xi_J]
constexpr uint32_t kIdescHalf = idesc_tf32(128, 128);
constexpr uint32_t kIdescBf16 = idesc_bf16(128, 256);
constexpr uint32_t kIdescBf16Half = idesc_bf16(128, 128);
// epilogue staging (reuses the tile region once every MMA has retired): the complex
// tile S and, for a diagonal tile, the ri block T1; rows padded to 129 elements so that
// a warp reading a column (lanes = rows) hits distinct banks
constexpr int kLd = kTile + 1;
constexpr int kT1Bytes = kTile * kLd * 4;
constexpr int kSOff = (kT1Bytes + 15) & ~15;
static_assert(kSOff + kTile * kLd * 8 <= kTiles, "epilogue staging exceeds the tile region");
static_assert(kTiles + 1024 + 256 <= 232448, "shared memory per CTA");

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

// Convert output chunks [c0, c1) of one row of a 128-row raw box (interleaved complex,
// 16 per row) into the planar rows of two destination tiles (re -> dre row rr, im ->
// dim row ri): FP32 (3xTF32) [hi 16 | lo 16] TF32 with chunks of 4 complex (c < 4),
// TF32 [hi 16] only, BF16 16 values in the first 32 bytes of the row with chunks of 8
// complex (c < 2).
__device__ __forceinline__ void convert_row(const char* raw, int r, char* dre, int rr, char* dim, int ri, int prec,
                                            int c0, int c1) {
    if (prec == FM_PREC_BF16) {
        for (int h = c0; h < c1; ++h) {  // output chunk h: complex 8h .. 8h+7
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
    for (int q = c0; q < c1; ++q) {  // output chunk q: complex 4q .. 4q+3
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

// The 8 epilogue warps (256 threads) synchronise among themselves; warps 0 and 1 do
// not take part.
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

// R (rows gi, columns gj of the frame) from the staged tile S (complex, row stride
// kLd): an off-diagonal tile writes R_IJ and its conjugate mirror R_JI, a diagonal tile
// its upper triangle and the conjugate of it below the diagonal (R exactly Hermitian).
// Warp w (0..7) takes rows w, w + 8, ...; lanes run along a row of R, so every store of
// a warp covers 32 consecutive elements.
__device__ __forceinline__ void write_tile(const float2* S, float2* __restrict__ R, int M, int i0, int j0, bool diag,
                                           int w, int lane) {
    for (int r = w; r < kTile; r += 8) {
        const int gi = i0 + r;
        if (gi >= M) break;
        for (int c = lane; c < kTile; c += 32) {
            const int gj = j0 + c;
            if (gj >= M) break;
            float2 v;
            if (!diag || c >= r) {
                v = S[r * kLd + c];
            } else {
                const float2 u = S[c * kLd + r];
                v = make_float2(u.x, -u.y);
            }
            R[(int64_t)gi * M + gj] = v;
        }
    }
    if (diag) return;
    // mirror: row gj of R holds conj(R_IJ[., c]); lanes run along the tile's rows
    for (int c = w; c < kTile; c += 8) {
        const int gj = j0 + c;
        if (gj >= M) break;
        for (int r = lane; r < kTile; r += 32) {
            const int gi = i0 + r;
            if (gi >= M) break;
            const float2 u = S[r * kLd + c];
            R[(int64_t)gj * M + gi] = make_float2(u.x, -u.y);
        }
    }
}

__global__ void __launch_bounds__(kThreads, 1)
    cov_tc_kernel(const FrameDesc* __restrict__ descs, const CUtensorMap* __restrict__ tmaps,
                  const CovItem* __restrict__ items, float2* __restrict__ partials, int* __restrict__ counters) {
    pdl_enter();
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char* raw = base;                              // kNRaw x {A, B}
    unsigned char* conv = base + kNRaw * kRawStage;         // kNConv x {Ar, Ai, B}
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + kTiles);
    uint64_t* raw_full = bars;                 // [kNRaw]
    uint64_t* raw_empty = bars + kNRaw;        // [kNRaw]
    uint64_t* conv_full = bars + 2 * kNRaw;    // [kNConv]
    uint64_t* conv_empty = conv_full + kNConv;  // [kNConv]
    uint64_t* acc_full = conv_empty + kNConv;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_full + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(acc_full + 2);
    int* s_flags = reinterpret_cast<int*>(acc_full + 3);  // [0] epilogue ok, [1] last part

    const CovItem it = items[blockIdx.x];
    const FrameDesc* dp = descs + it.frame;
    const int M = dp->M, T = dp->T, prec = dp->prec;  // prec is uniform over the CTA
    const bool diag = (it.ti == it.tj);
    const int i0 = it.ti * kTile, j0 = it.tj * kTile;
    const int s0 = it.s0, nstages = it.s1 - it.s0;
    const CUtensorMap* tm = tmaps + it.frame;
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
                tma_load_2d(dst, tm, (s0 + s) * 32, i0, &raw_full[slot]);
                if (!diag) tma_load_2d(dst + kRawBox, tm, (s0 + s) * 32, j0, &raw_full[slot]);
            }
            // drain: the last loads must land before the CTA may exit
            for (int s = max(0, nstages - kNRaw); s < nstages; ++s)
                mbar_wait(&raw_full[s % kNRaw], (uint32_t)(s / kNRaw) & 1u, abort_flag);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------- MMA issuer --
        // off-diagonal: d_top = [rr | ri] (N = 256), d_bot = [ir | ii] (N = 256);
        // diagonal: d_top = [rr | ri] (N = 256), d_bot = ii (N = 128), A = halves of B
        if (lane == 0) {
            const uint32_t d_top = tmem, d_bot = tmem + 256;
            const uint32_t idesc_bot = diag ? kIdescHalf : kIdesc;
            for (int s = 0; s < nstages; ++s) {
                const int slot = s % kNConv;
                const uint32_t ph = (uint32_t)(s / kNConv) & 1u;
                if (!mbar_wait(&conv_full[slot], ph, abort_flag)) break;
                tc_fence_after();
                unsigned char* cv = conv + slot * kConvStage;
                const uint32_t bb = sa(cv + 2 * kConvA);
                const uint32_t ar = diag ? bb : sa(cv), ai = diag ? bb + kConvA : sa(cv + kConvA);
                const uint32_t bbot = diag ? bb + kConvA : bb;  // B of d_bot: [Xr; Xi] or Xi alone
                if (prec == FM_PREC_BF16) {  // one K = 16 step covers the stage's 16 snapshots
                    const uint32_t acc0 = s > 0 ? 1u : 0u;
                    mma_bf16(d_top, desc_sw128(ar), desc_sw128(bb), kIdescBf16, acc0);
                    mma_bf16(d_bot, desc_sw128(ai), desc_sw128(bbot), diag ? kIdescBf16Half : kIdescBf16, acc0);
                } else {
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk) {
                        const uint32_t acc0 = (s > 0 || kk > 0) ? 1u : 0u;
                        const uint64_t b_hi = desc_sw128(bb + 32 * kk), b_lo = desc_sw128(bb + 64 + 32 * kk);
                        const uint64_t c_hi = desc_sw128(bbot + 32 * kk), c_lo = desc_sw128(bbot + 64 + 32 * kk);
                        const uint64_t r_hi = desc_sw128(ar + 32 * kk), r_lo = desc_sw128(ar + 64 + 32 * kk);
                        const uint64_t i_hi = desc_sw128(ai + 32 * kk), i_lo = desc_sw128(ai + 64 + 32 * kk);
                        mma_tf32(d_top, r_hi, b_hi, kIdesc, acc0);
                        mma_tf32(d_bot, i_hi, c_hi, idesc_bot, acc0);
                        if (prec == FM_PREC_FP32) {  // 3xTF32: + hi*lo + lo*hi
                            mma_tf32(d_top, r_hi, b_lo, kIdesc, 1u);
                            mma_tf32(d_top, r_lo, b_hi, kIdesc, 1u);
                            mma_tf32(d_bot, i_hi, c_lo, idesc_bot, 1u);
                            mma_tf32(d_bot, i_lo, c_hi, idesc_bot, 1u);
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
        // off-diagonal: thread r < 128 converts row r of A into Ar, Ai; thread r >= 128
        // row r - 128 of B into [Br; Bi].  Diagonal: only B is converted, thread r takes
        // half of the output chunks of row r % 128.
        const int r = threadIdx.x - 64;  // 0..255
        const bool is_b = r >= kTile;
        const int rr = r & (kTile - 1);
        const int nch = (prec == FM_PREC_BF16) ? 2 : 4;
        const int c0 = diag ? (is_b ? nch / 2 : 0) : 0, c1 = diag ? (is_b ? nch : nch / 2) : nch;
        for (int s = 0; s < nstages; ++s) {
            const int rs = s % kNRaw, cs = s % kNConv;
            if (!mbar_wait(&raw_full[rs], (uint32_t)(s / kNRaw) & 1u, abort_flag)) break;
            if (!mbar_wait(&conv_empty[cs], ((uint32_t)(s / kNConv) & 1u) ^ 1u, abort_flag)) break;
            const char* rawA = reinterpret_cast<const char*>(raw + rs * kRawStage);
            char* cv = reinterpret_cast<char*>(conv + cs * kConvStage);
            if (diag)
                convert_row(rawA, rr, cv + 2 * kConvA, rr, cv + 2 * kConvA, 128 + rr, prec, c0, c1);
            else if (!is_b)
                convert_row(rawA, rr, cv, rr, cv + kConvA, rr, prec, 0, nch);                          // Ar, Ai
            else
                convert_row(rawA + kRawBox, rr, cv + 2 * kConvA, rr, cv + 2 * kConvA, 128 + rr, prec, 0, nch);  // B
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(&conv_full[cs]);
            mbar_arrive(&raw_empty[rs]);
        }
        // ----- epilogue: TMEM -> S (shared) -> R.  A warp reads only its TMEM lane
        // quadrant q = warp % 4 (rows 32 q + lane) and columns [64 h, 64 h + 64),
        // h = 0 for warps 2-5.  `ok` is made uniform over the 8 warps before any of
        // their barriers (tcgen05.ld below is .sync.aligned).
        const bool wok = __all_sync(0xffffffffu, mbar_wait(acc_full, 0u, abort_flag));
        if (threadIdx.x == 64) s_flags[0] = 1;
        epi_sync();
        if (!wok && lane == 0) s_flags[0] = 0;
        epi_sync();
        const bool ok = s_flags[0] != 0;
        tc_fence_after();
        const int ew = warp - 2;  // 0..7
        if (ok) {
            float* T1 = reinterpret_cast<float*>(base);
            float2* S = reinterpret_cast<float2*>(base + kSOff);
            const int q = warp & 3;
            const int row = 32 * q + lane;
            const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16);
            const float invT = (float)(1.0 / (double)T);
            const int h = (warp - 2) >> 2;
            if (diag) {  // the ri block first: Im R_II = (ri^T - ri) / T (four TMEM loads per wait)
                uint32_t ri[4][16];
#pragma unroll
                for (int b = 0; b < 4; ++b) tmem_ld16(tl + 128 + 64 * h + 16 * b, ri[b]);
                tmem_wait_ld();
#pragma unroll
                for (int b = 0; b < 4; ++b)
#pragma unroll
                    for (int c = 0; c < 16; ++c) T1[row * kLd + 64 * h + 16 * b + c] = __uint_as_float(ri[b][c]);
                epi_sync();
            }
            for (int c2 = 64 * h; c2 < 64 * h + 64; c2 += 32) {  // two 16-column chunks per TMEM wait
                uint32_t rr_[2][16], a1[2][16], a2[2][16], riv[2][16];
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    const int cc = c2 + 16 * b;
                    tmem_ld16(tl + cc, rr_[b]);
                    if (diag) {
                        tmem_ld16(tl + 256 + cc, a1[b]);  // ii
                    } else {
                        tmem_ld16(tl + 256 + cc, a2[b]);  // ir
                        tmem_ld16(tl + 384 + cc, a1[b]);  // ii
                        tmem_ld16(tl + 128 + cc, riv[b]);
                    }
                }
                tmem_wait_ld();
#pragma unroll
                for (int b = 0; b < 2; ++b)
#pragma unroll
                    for (int c = 0; c < 16; ++c) {
                        const int col = c2 + 16 * b + c;
                        const float re = (__uint_as_float(rr_[b][c]) + __uint_as_float(a1[b][c])) * invT;
                        float im;
                        if (diag)
                            im = (col == row) ? 0.f : (T1[col * kLd + row] - T1[row * kLd + col]) * invT;
                        else
                            im = (__uint_as_float(a2[b][c]) - __uint_as_float(riv[b][c])) * invT;
                        S[row * kLd + col] = make_float2(re, im);
                    }
            }
            epi_sync();
            if (it.split < 0) {
                write_tile(S, dp->R, M, i0, j0, diag, ew, lane);
            } else {
                // partial tile -> its slot (row-major 128 x 128); the last part adds them all
                float2* __restrict__ mine = partials + (int64_t)(it.first + it.k) * kTile * kTile;
                for (int rw = ew; rw < kTile; rw += 8)
                    for (int c = lane; c < kTile; c += 32) mine[rw * kTile + c] = S[rw * kLd + c];
                __threadfence();
                epi_sync();
                if (threadIdx.x == 64) s_flags[1] = (atomicAdd(&counters[it.split], 1) == it.nparts - 1) ? 1 : 0;
                epi_sync();
                if (s_flags[1]) {
                    __threadfence();
                    const float2* __restrict__ first = partials + (int64_t)it.first * kTile * kTile;
                    for (int rw = ew; rw < kTile; rw += 8)
                        for (int c = lane; c < kTile; c += 32) {
                            float2 acc = make_float2(0.f, 0.f);
                            for (int k = 0; k < it.nparts; ++k) {
                                const float2 v = __ldcg(first + ((int64_t)k * kTile + rw) * kTile + c);
                                acc.x += v.x;
                                acc.y += v.y;
                            }
                            S[rw * kLd + c] = acc;
                        }
                    epi_sync();
                    write_tile(S, dp->R, M, i0, j0, diag, ew, lane);
                    if (threadIdx.x == 64) counters[it.split] = 0;  // ready for the next run
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

cudaError_t launch_covariance_tc(const FrameDesc* d, const void* tmaps, const CovItem* items, int n_items,
                                 float2* partials, int* counters, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(cov_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    count_launch();
    launch_pdl(cov_tc_kernel, dim3(n_items), dim3(kThreads), (size_t)(kSmemBytes), s, d, reinterpret_cast<const CUtensorMap*>(tmaps), items,
                                                        partials, counters);
    return cudaGetLastError();
}

}  // namespace fm

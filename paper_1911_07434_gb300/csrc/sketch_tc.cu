// sketch_tc.cu -- the sketch products C = R V (Sec. III, Alg. 1 / Alg. 2, Eq. 11) on
// the 5th-generation tensor cores, FP32 accumulation.
//
// Real formulation on interleaved complex rows: a row of R is read as 2M FP32
// values [Rr_0, Ri_0, Rr_1, Ri_1, ...], and every column j of V becomes two B rows
//   [Vr_0, -Vi_0, Vr_1, -Vi_1, ...] -> Re C[., j],   [Vi_0, Vr_0, Vi_1, Vr_1, ...] -> Im C[., j],
// so one real GEMM D = R_rows B^T (K = 2M, N = 2 l_pad) gives C.
//
// Two kernels (sketch_bprep_kernel writes the B rows of both, and generates Omega for the
// projection variant's first product):
// * sketch_tc_kernel, TF32 operands, one MMA per product: R streams from HBM by
//   TMA straight into the 128-byte-swizzled K-major layout the MMA reads (the tensor
//   core takes the TF32 part of each FP32 value), B rows rounded to TF32.  It takes
//   every product of a TF32 / BF16 frame.
// * sketch_split_kernel, FP32 accuracy, three TF32 MMAs per product (hi*hi + hi*lo
//   + lo*hi, as the covariance does): every product of an FP32 frame (the core
//   matrix depends on the last basis V, so every product that leads to it is kept at
//   FP32 accuracy).  R arrives raw by TMA in the swizzled layout the MMA reads (128
//   rows x 32 FP32 per stage) and serves as the hi operand as it is: the tensor core
//   truncates each FP32 operand to TF32 (checked on GB300).  Four converter warps
//   write only the lo tile, x - trunc_tf32(x) rounded to TF32, at the same swizzled
//   positions; the B rows come pre-split in [hi 16 | lo 16] chunks (hi = rn_tf32).
//
// One CTA per 128 rows of R of one frame: warp 0 issues TMA loads (ring of stages),
// warp 1 allocates TMEM and issues the MMAs (one thread), warps 2-5 convert (split
// kernel) and run the epilogue.  Shared memory is sized for the launch's largest l
// so that two CTAs fit on an SM.  Every mbarrier wait is bounded and records
// FM_ERR_TIMEOUT on expiry.
#include "tc_common.cuh"

namespace fm {
namespace {

using namespace tc;

constexpr int kRows = 128;
constexpr int kTileA = kRows * 128;    // 16 KB: 128 rows x 128 B (32 FP32, or [hi 16 | lo 16] TF32)
constexpr int kThreads = 192;
constexpr int kSmemPerCta = 113 * 1024;  // two CTAs per SM (228 KB, 1 KB reserved per CTA)
constexpr int kSmemExtra = 1024 + 256;   // 1024-B alignment slack + barriers
constexpr uint32_t kTmemCols = 128;

// Ring geometry for B tiles of nb_max rows (nb_max = 2 l_pad of the launch's largest l).
__host__ __device__ constexpr int plain_stage(int nb_max) { return kTileA + nb_max * 128; }
__host__ __device__ constexpr int plain_nstages(int nb_max) {
    return 4 * plain_stage(nb_max) + kSmemExtra <= kSmemPerCta ? 4 : 3;
}
// Split kernel: a ring of stages [B chunk 0 | B chunk 1 (nb_max x 128 B each) | raw A 16 KB]
// (32 FP32 of K per stage) as deep as two CTAs per SM allow (at most 6), and two lo tiles
// where three stages still fit beside them (else one: the ring depth matters more).
__host__ __device__ constexpr int split_stage(int nb_max) { return 2 * nb_max * 128 + kTileA; }
__host__ __device__ constexpr int split_nlo(int nb_max) {
    return 3 * split_stage(nb_max) + 2 * kTileA + kSmemExtra <= kSmemPerCta ? 2 : 1;
}
__host__ __device__ constexpr int split_nraw(int nb_max) {
    int n = 6;
    while (n > 2 && n * split_stage(nb_max) + split_nlo(nb_max) * kTileA + kSmemExtra > kSmemPerCta) --n;
    return n;
}
__host__ __device__ constexpr int split_smem(int nb_max) {
    return split_nraw(nb_max) * split_stage(nb_max) + split_nlo(nb_max) * kTileA + kSmemExtra;
}
static_assert(split_nraw(2 * kLMax) >= 2 && split_smem(2 * kLMax) <= kSmemPerCta, "split ring too large");
static_assert(plain_nstages(2 * kLMax) * plain_stage(2 * kLMax) + kSmemExtra <= kSmemPerCta, "ring too large");

// B rows of pass `pass` from 64 rows of V per block.  Plain layout (2 l_pad rows x
// 2M): TF32-rounded [Vr, -Vi] and [Vi, Vr] rows.  Split layout (2 l_pad rows x 32
// ceil(2M/16)): chunk c of 16 values stored as [hi 16 | lo 16], hi = rn_tf32(v),
// lo = rn_tf32(v - hi), the last chunk's padding (m >= M) written as zeros.  The V
// tile (64 x l complex, contiguous in V) is staged in shared memory with coalesced
// loads; for the projection variant's first product it is generated instead (the
// Gaussian test matrix Omega of Alg. 2, also written to V, which holds Pi for the
// core matrix when t = 0).  Consecutive threads then write consecutive 16-byte
// pieces (split) or complex pairs (plain) of a B row segment.
constexpr int kBpRows = 64;
constexpr int kBpThreads = 256;
constexpr int kBpFill = kBpRows * kLMax / kBpThreads;  // tile entries per thread at most
constexpr int kBpLd = kLMax + 1;  // odd row stride (in float2) against bank conflicts
__global__ void __launch_bounds__(kBpThreads) sketch_bprep_kernel(const FrameDesc* __restrict__ descs, int pass) {
    pdl_enter();
    __shared__ float2 vt[kBpRows * kBpLd];
    const FrameDesc* dp = descs + blockIdx.y;
    if (!dp->sketch_tc || pass > dp->t || !sketch_on_tc(dp->method, pass)) return;
    if (pass > 0 && dp->bsk_orth_nc > 0) return;  // written by the orthonormalisation
    const int M = dp->M, l = dp->l, lp = sketch_tc_lpad(l);
    const int m0 = blockIdx.x * kBpRows;
    if (m0 >= M) return;
    const int rows = min(kBpRows, M - m0);
    const bool gen = pass == 0 && dp->method == FM_RAND_PROJECTION;
    // every load (or Omega entry) of the thread in flight at once, then into shared memory
    float2 vv[kBpFill];
#pragma unroll
    for (int u = 0; u < kBpFill; ++u) {
        const int e = threadIdx.x + kBpThreads * u;
        vv[u] = make_float2(0.f, 0.f);
        if (e < rows * l) {
            if (gen) {
                const int r = e / l;
                vv[u] = gaussian_entry(dp->seed, dp->frame_id, m0 + r, e - r * l);
            } else {
                vv[u] = dp->V[(int64_t)m0 * l + e];
            }
        }
    }
#pragma unroll
    for (int u = 0; u < kBpFill; ++u) {
        const int e = threadIdx.x + kBpThreads * u;
        if (e < kBpRows * l) {
            const int r = e / l;
            vt[r * kBpLd + (e - r * l)] = vv[u];
            if (gen && e < rows * l) dp->V[(int64_t)m0 * l + e] = vv[u];
        }
    }
    __syncthreads();
    const int nrow = 2 * lp;
    if (!sketch_split(dp->prec, dp->t, pass)) {
        // one complex entry m per thread: (re row) [Vr, -Vi], (im row) [Vi, Vr] at 2m
        const int64_t rowlen = 2 * (int64_t)M;
        for (int t = threadIdx.x; t < nrow * kBpRows; t += kBpThreads) {
            const int R = t / kBpRows, r = t - R * kBpRows;
            if (r >= rows) continue;
            const int j = R >> 1;
            const float2 v = j < l ? vt[r * kBpLd + j] : make_float2(0.f, 0.f);
            const float a = (R & 1) ? v.y : v.x, b = (R & 1) ? v.x : -v.y;
            *reinterpret_cast<float2*>(dp->Bsk + R * rowlen + 2 * (int64_t)(m0 + r)) =
                make_float2(__uint_as_float(tf32_rn(a)), __uint_as_float(tf32_rn(b)));
        }
        return;
    }
    // split: a row segment is 8 chunks x 8 pieces of 16 bytes; piece p < 4 holds the hi
    // values 4p .. 4p+3 of its chunk (entries m = 8c + 2p, 8c + 2p + 1), p >= 4 their lo
    const int64_t rowlen = sketch_split_rowlen(M);
    const int nchunks = (2 * M + 15) / 16, c0 = m0 / 8;
    for (int t = threadIdx.x; t < nrow * 64; t += kBpThreads) {
        const int R = t >> 6, cc = (t >> 3) & 7, p = t & 7;
        const int c = c0 + cc;
        if (c >= nchunks) continue;
        const int j = R >> 1, ra = 8 * cc + 2 * (p & 3);
        float2 va = make_float2(0.f, 0.f), vb = va;
        if (j < l) {
            va = vt[ra * kBpLd + j];
            vb = vt[(ra + 1) * kBpLd + j];
        }
        const float x[4] = {(R & 1) ? va.y : va.x, (R & 1) ? va.x : -va.y, (R & 1) ? vb.y : vb.x,
                            (R & 1) ? vb.x : -vb.y};
        uint4 o;
        uint32_t* ov = reinterpret_cast<uint32_t*>(&o);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t hi = tf32_rn(x[u]);
            ov[u] = p < 4 ? hi : tf32_rn(x[u] - __uint_as_float(hi));
        }
        *reinterpret_cast<uint4*>(dp->Bsk + R * rowlen + 32 * (int64_t)c + 4 * p) = o;
    }
}

struct Ring {
    uint64_t* full;   // [ns] TMA -> MMA
    uint64_t* empty;  // [ns] MMA -> TMA
    uint64_t* acc_full;
    uint32_t* tmem_slot;
    volatile int* abort_flag;
};

__device__ __forceinline__ Ring ring_at(unsigned char* p, int ns) {
    Ring r;
    uint64_t* bars = reinterpret_cast<uint64_t*>(p);
    r.full = bars;
    r.empty = bars + ns;
    r.acc_full = bars + 2 * ns;
    r.tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * ns + 1);
    r.abort_flag = reinterpret_cast<volatile int*>(bars + 2 * ns + 2);
    return r;
}

// Epilogue of warps 2-5: TMEM lane quadrant warp % 4 = rows 32 q + lane of the tile;
// accumulator column 2j = Re C[., j], 2j + 1 = Im C[., j].
__device__ __forceinline__ void store_c(const FrameDesc* dp, const Ring& rg, uint32_t tmem, int r0, int nb, int warp,
                                        int lane) {
    const bool ok = __all_sync(0xffffffffu, mbar_wait(rg.acc_full, 0u, rg.abort_flag));
    tc_fence_after();
    if (ok) {
        const int M = dp->M, l = dp->l;
        const int q = warp & 3;
        const int gr = r0 + 32 * q + lane;
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

__device__ __forceinline__ uint32_t tmem_setup(const Ring& rg, int ns, const CUtensorMap* ta, const CUtensorMap* tb,
                                               int full_count) {
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        for (int s = 0; s < ns; ++s) {
            mbar_init(&rg.full[s], (uint32_t)full_count);
            mbar_init(&rg.empty[s], 1);
        }
        mbar_init(rg.acc_full, 1);
        *rg.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        tmap_acquire(ta);
        tmap_acquire(tb);
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa(rg.tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    return *rg.tmem_slot;
}

__device__ __forceinline__ void tmem_teardown(const FrameDesc* dp, const Ring& rg, uint32_t tmem) {
    __syncthreads();
    if (*rg.abort_flag && threadIdx.x == 0) set_status(dp->status, FM_ERR_TIMEOUT);
    if ((threadIdx.x >> 5) == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

__global__ void __launch_bounds__(kThreads, 2)
    sketch_tc_kernel(const FrameDesc* __restrict__ descs, const CUtensorMap* __restrict__ tmA,
                     const CUtensorMap* __restrict__ tmB, int pass, int nb_max) {
    pdl_enter();
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int ns = plain_nstages(nb_max), stage = plain_stage(nb_max);
    const FrameDesc* dp = descs + blockIdx.y;
    // frames whose last product is done (pass > t) keep their C
    if (!dp->sketch_tc || pass > dp->t || !sketch_on_tc(dp->method, pass) || sketch_split(dp->prec, dp->t, pass))
        return;
    const int M = dp->M, nb = 2 * sketch_tc_lpad(dp->l);
    const int r0 = blockIdx.x * kRows;
    if (r0 >= M) return;
    const int nstages = (2 * M + 31) / 32;
    const CUtensorMap* ta = tmA + blockIdx.y;
    const CUtensorMap* tb = tmB + blockIdx.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const Ring rg = ring_at(base + ns * stage, ns);
    const uint32_t tmem = tmem_setup(rg, ns, ta, tb, 1);

    if (warp == 0) {
        if (lane == 0) {
            const uint32_t bytes = (uint32_t)kTileA + (uint32_t)nb * 128u;
            for (int s = 0; s < nstages; ++s) {
                const int slot = s % ns;
                if (!mbar_wait(&rg.empty[slot], ((uint32_t)(s / ns) & 1u) ^ 1u, rg.abort_flag)) break;
                unsigned char* dst = base + slot * stage;
                mbar_expect_tx(&rg.full[slot], bytes);
                tma_load_2d(dst, ta, s * 32, r0, &rg.full[slot]);
                tma_load_2d(dst + kTileA, tb, s * 32, 0, &rg.full[slot]);
            }
            for (int s = max(0, nstages - ns); s < nstages; ++s)
                mbar_wait(&rg.full[s % ns], (uint32_t)(s / ns) & 1u, rg.abort_flag);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_tf32(128, (uint32_t)nb);
            for (int s = 0; s < nstages; ++s) {
                const int slot = s % ns;
                if (!mbar_wait(&rg.full[slot], (uint32_t)(s / ns) & 1u, rg.abort_flag)) break;
                tc_fence_after();
                const uint32_t a = sa(base + slot * stage), b = a + kTileA;
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)  // 32 values per row = four K = 8 steps of 32 bytes
                    mma_tf32(tmem, desc_sw128(a + 32 * kk), desc_sw128(b + 32 * kk), idesc, (s > 0 || kk > 0) ? 1u : 0u);
                mma_commit(&rg.empty[slot]);
            }
            mma_commit(rg.acc_full);
            mbar_wait(rg.acc_full, 0u, rg.abort_flag);
        }
    } else {
        store_c(dp, rg, tmem, r0, nb, warp, lane);
    }
    tmem_teardown(dp, rg, tmem);
}

// Split kernel, two-level sum: the MMAs of each group of kGroup stages accumulate in
// one of two TMEM buffers (columns 0 and 128), and warps 2-5 add every finished group
// into FP32 registers, as the CUDA-core sketch sums per chunk and then across chunks.
// A single accumulator over all the MMAs of a row would carry the tensor core's
// accumulation error of every step (measured: 2.4x the projector error at M = 1024).
constexpr int kGroup = 4;                 // stages (32 values of K each) per group
constexpr uint32_t kSplitTmemCols = 256;  // two accumulators of up to 128 columns

template <int NB>
__global__ void __launch_bounds__(kThreads, 2)
    sketch_split_kernel(const FrameDesc* __restrict__ descs, const CUtensorMap* __restrict__ tmA,
                        const CUtensorMap* __restrict__ tmB, int pass) {
    pdl_enter();
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    constexpr int nr = split_nraw(NB);
    constexpr int nlo = split_nlo(NB);
    constexpr int stage = split_stage(NB);
    constexpr int b1_off = NB * 128, a_off = 2 * NB * 128;  // stage: [B chunk 0 | B chunk 1 | raw A]
    const FrameDesc* dp = descs + blockIdx.y;
    // frames whose last product is done (pass > t) keep their C
    if (!dp->sketch_tc || pass > dp->t || !sketch_on_tc(dp->method, pass) || !sketch_split(dp->prec, dp->t, pass))
        return;
    const int M = dp->M, l = dp->l, nb = 2 * sketch_tc_lpad(l);
    const int r0 = blockIdx.x * kRows;
    if (r0 >= M) return;
    const int nst = (2 * M + 31) / 32;  // stages of 32 FP32 of K (the last one zero-filled past 2M)
    const int ngroups = (nst + kGroup - 1) / kGroup;
    const CUtensorMap* ta = tmA + blockIdx.y;
    const CUtensorMap* tb = tmB + blockIdx.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // layout: nr stages, nlo lo tiles, barriers
    unsigned char* lo_tiles = base + nr * stage;
    uint64_t* bars = reinterpret_cast<uint64_t*>(lo_tiles + nlo * kTileA);
    uint64_t* full = bars;                 // [nr] raw A + B chunks landed (TMA)
    uint64_t* empty = bars + nr;           // [nr] MMA done with the stage
    uint64_t* conv_full = bars + 2 * nr;   // [2] lo tile written (128 converter arrivals)
    uint64_t* conv_empty = conv_full + 2;  // [2] MMA done with the lo tile
    uint64_t* acc_ready = conv_full + 4;   // [2] group committed -> drain
    uint64_t* acc_free = conv_full + 6;    // [2] group drained (128 arrivals) -> MMA
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(conv_full + 8);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(conv_full + 9);

    if (threadIdx.x == 0) {
        for (int i = 0; i < nr; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&conv_full[i], 128);
            mbar_init(&conv_empty[i], 1);
            mbar_init(&acc_ready[i], 1);
            mbar_init(&acc_free[i], 128);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        tmap_acquire(ta);
        tmap_acquire(tb);
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa(tmem_slot)),
                     "r"(kSplitTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            const uint32_t bytes = (uint32_t)kTileA + 2u * (uint32_t)nb * 128u;
            for (int s = 0; s < nst; ++s) {
                const int slot = s % nr;
                if (!mbar_wait(&empty[slot], ((uint32_t)(s / nr) & 1u) ^ 1u, abort_flag)) break;
                unsigned char* st = base + slot * stage;
                mbar_expect_tx(&full[slot], bytes);
                tma_load_2d(st + a_off, ta, s * 32, r0, &full[slot]);
                tma_load_2d(st, tb, s * 64, 0, &full[slot]);
                tma_load_2d(st + b1_off, tb, s * 64 + 32, 0, &full[slot]);
            }
            for (int s = max(0, nst - nr); s < nst; ++s)
                mbar_wait(&full[s % nr], (uint32_t)(s / nr) & 1u, abort_flag);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_tf32(128, (uint32_t)nb);
            for (int s = 0; s < nst; ++s) {
                const int slot = s % nr, g = s / kGroup, buf = g & 1, sg = s % kGroup;
                const uint32_t d = tmem + 128u * (uint32_t)buf;
                if (sg == 0 && g >= 2) {  // buffer buf still holds group g - 2 until it is drained
                    if (!mbar_wait(&acc_free[buf], (uint32_t)((g >> 1) + 1) & 1u, abort_flag)) break;
                }
                if (!mbar_wait(&full[slot], (uint32_t)(s / nr) & 1u, abort_flag)) break;
                tc_fence_after();
                const uint32_t st = sa(base + slot * stage), a = st + a_off, alo = sa(lo_tiles + (s % nlo) * kTileA);
                // the raw (hi) products first, while the converters write the lo tile; K = 8
                // steps, the tensor core truncating raw A to TF32
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const uint32_t bt = st + (kk >> 1) * b1_off + 32 * (kk & 1);
                    const uint64_t a_hi = desc_sw128(a + 32 * kk);
                    mma_tf32(d, a_hi, desc_sw128(bt), idesc, (sg > 0 || kk > 0) ? 1u : 0u);
                    mma_tf32(d, a_hi, desc_sw128(bt + 64), idesc, 1u);
                }
                if (!mbar_wait(&conv_full[s % nlo], (uint32_t)(s / nlo) & 1u, abort_flag)) break;
                tc_fence_after();
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const uint32_t bt = st + (kk >> 1) * b1_off + 32 * (kk & 1);
                    mma_tf32(d, desc_sw128(alo + 32 * kk), desc_sw128(bt), idesc, 1u);
                }
                mma_commit(&conv_empty[s % nlo]);
                mma_commit(&empty[slot]);
                if (sg == kGroup - 1 || s == nst - 1) mma_commit(&acc_ready[buf]);
            }
            // all MMAs retired before dealloc: the last group's commit tracks every earlier MMA
            mbar_wait(&acc_ready[(ngroups - 1) & 1], (uint32_t)((ngroups - 1) >> 1) & 1u, abort_flag);
        }
    } else {
        // converters + two-level sum.  Thread t = 0..127 owns row t of the stage: the lo
        // parts x - trunc_tf32(x), rounded to TF32, of its 8 raw 16-byte chunks go to the
        // same swizzled positions of the lo tile (lanes = rows: every 8-lane phase touches
        // eight distinct 16-byte bank groups).  Sum: the same thread owns TMEM lane t (its
        // warp's lane quadrant) and keeps the row's NB accumulator columns in registers.
        const int q4 = warp & 3, t = 32 * q4 + lane;
        const uint32_t tl = tmem + ((uint32_t)(32 * q4) << 16);
        float sum[NB];
#pragma unroll
        for (int j = 0; j < NB; ++j) sum[j] = 0.f;
        bool ok = true;
        int gd = 0;  // next group to drain
        auto drain = [&](int g) {
            const int buf = g & 1;
            ok = ok && __all_sync(0xffffffffu, mbar_wait(&acc_ready[buf], (uint32_t)(g >> 1) & 1u, abort_flag));
            if (!ok) return;
            tc_fence_after();
#pragma unroll
            for (int c0 = 0; c0 < NB; c0 += 48) {  // up to three 16-column loads per wait
                uint32_t v[48];
#pragma unroll
                for (int u = 0; u < 48; u += 16)
                    if (c0 + u < NB) tmem_ld16(tl + 128u * (uint32_t)buf + (uint32_t)(c0 + u), *reinterpret_cast<uint32_t(*)[16]>(v + u));
                tmem_wait_ld();
#pragma unroll
                for (int u = 0; u < 48; ++u)
                    if (c0 + u < NB) sum[c0 + u] += __uint_as_float(v[u]);
            }
            tc_fence_before();
            mbar_arrive(&acc_free[buf]);
        };
        for (int s = 0; s < nst && ok; ++s) {
            const int slot = s % nr;
            if (!__all_sync(0xffffffffu, mbar_wait(&full[slot], (uint32_t)(s / nr) & 1u, abort_flag))) {
                ok = false;
                break;
            }
            const unsigned char* raw = base + slot * stage + a_off;
            uint4 lo[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const uint4 v = *reinterpret_cast<const uint4*>(raw + swz(t, c));
                lo[c].x = tf32_rn(__uint_as_float(v.x) - __uint_as_float(v.x & 0xFFFFE000u));
                lo[c].y = tf32_rn(__uint_as_float(v.y) - __uint_as_float(v.y & 0xFFFFE000u));
                lo[c].z = tf32_rn(__uint_as_float(v.z) - __uint_as_float(v.z & 0xFFFFE000u));
                lo[c].w = tf32_rn(__uint_as_float(v.w) - __uint_as_float(v.w & 0xFFFFE000u));
            }
            // the MMAs of stage s - nlo are done with this lo tile
            if (!__all_sync(0xffffffffu, mbar_wait(&conv_empty[s % nlo], ((uint32_t)(s / nlo) & 1u) ^ 1u, abort_flag))) {
                ok = false;
                break;
            }
            unsigned char* lo_tile = lo_tiles + (s % nlo) * kTileA;
#pragma unroll
            for (int c = 0; c < 8; ++c) *reinterpret_cast<uint4*>(lo_tile + swz(t, c)) = lo[c];
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(&conv_full[s % nlo]);
            // the lo tile of stage s was free, so every MMA up to stage s - nlo has completed:
            // the groups that ended there are ready
            while (ok && gd < ngroups && min(gd * kGroup + kGroup - 1, nst - 1) + nlo <= s) drain(gd++);
        }
        while (ok && gd < ngroups) drain(gd++);
        const int gr = r0 + t;
        if (ok && gr < M) {
            float2* __restrict__ C = dp->C + (int64_t)gr * l;
#pragma unroll
            for (int j = 0; j < NB / 2; ++j)
                if (j < l) C[j] = make_float2(sum[2 * j], sum[2 * j + 1]);
        }
    }
    __syncthreads();
    if (*abort_flag && threadIdx.x == 0) set_status(dp->status, FM_ERR_TIMEOUT);
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kSplitTmemCols)
                     : "memory");
    }
}

}  // namespace

template <int NB>
cudaError_t launch_split(const FrameDesc* d, dim3 grid, int pass, const void* tmA, const void* tmB, cudaStream_t s) {
    static_assert(NB % 16 == 0 && NB <= 2 * kLMax, "B rows: 2 l_pad");
    const int smem = split_smem(NB);
    cudaError_t e = cudaFuncSetAttribute(sketch_split_kernel<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    count_launch();
    launch_pdl(sketch_split_kernel<NB>, dim3(grid), dim3(kThreads), (size_t)(smem), s, d, reinterpret_cast<const CUtensorMap*>(tmA),
                                                         reinterpret_cast<const CUtensorMap*>(tmB), pass);
    return cudaGetLastError();
}

size_t sketch_tc_smem_bytes(int max_l, bool split) {
    const int nb_max = 2 * sketch_tc_lpad(max_l);
    return split ? (size_t)split_smem(nb_max)
                 : (size_t)plain_nstages(nb_max) * plain_stage(nb_max) + kSmemExtra;
}

cudaError_t launch_sketch_tc(const FrameDesc* d, int n_frames, int max_M, int max_l, int pass, bool any_plain,
                             bool any_split, const void* tmA, const void* tmB, const void* tmA_split,
                             const void* tmB_split, cudaStream_t s, bool prep) {
    const int lp = sketch_tc_lpad(max_l), nb_max = 2 * lp;
    cudaError_t e = cudaSuccess;
    if (prep) {
        count_launch();
        launch_pdl(sketch_bprep_kernel, dim3(dim3((unsigned)((max_M + kBpRows - 1) / kBpRows), n_frames)), dim3(kBpThreads), (size_t)(0), s, d, pass);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const dim3 grid((unsigned)((max_M + kRows - 1) / kRows), n_frames);
    if (any_plain) {
        const int smem = (int)sketch_tc_smem_bytes(max_l, false);
        e = cudaFuncSetAttribute(sketch_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        count_launch();
        launch_pdl(sketch_tc_kernel, dim3(grid), dim3(kThreads), (size_t)(smem), s, d, reinterpret_cast<const CUtensorMap*>(tmA),
                                                      reinterpret_cast<const CUtensorMap*>(tmB), pass, nb_max);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (any_split) {
        switch (nb_max) {  // 2 l_pad, l_pad a multiple of 8 up to kLMax
            case 16: return launch_split<16>(d, grid, pass, tmA, tmB_split, s);
            case 32: return launch_split<32>(d, grid, pass, tmA, tmB_split, s);
            case 48: return launch_split<48>(d, grid, pass, tmA, tmB_split, s);
            case 64: return launch_split<64>(d, grid, pass, tmA, tmB_split, s);
            case 80: return launch_split<80>(d, grid, pass, tmA, tmB_split, s);
            default: return launch_split<96>(d, grid, pass, tmA, tmB_split, s);
        }
    }
    return e;
}

}  // namespace fm

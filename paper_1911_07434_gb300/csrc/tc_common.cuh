// tc_common.cuh -- inline-PTX helpers shared by the tensor-core kernels:
// mbarriers (bounded waits), TMA tile loads, TF32 rounding, tcgen05 shared-memory
// and instruction descriptors, MMA issue/commit, TMEM loads and fences.
#pragma once

#include <cuda.h>

#include "fm_internal.cuh"

namespace fm {
namespace tc {

constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz: bound on every mbarrier wait

__device__ __forceinline__ uint32_t sa(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sa(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sa(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sa(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(sa(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: false (and *abort set) if the phase did not complete within
// limit_cycles SM clocks (or another thread of the CTA gave up first).
__device__ __forceinline__ bool mbar_wait_limit(uint64_t* b, uint32_t parity, volatile int* abort,
                                                long long limit_cycles) {
    if (mbar_test(b, parity)) return true;
    const long long t0 = clock64();
    while (true) {
        if (mbar_test(b, parity)) return true;
        if (*abort) return false;
        if (clock64() - t0 > limit_cycles) {
            *abort = 1;
            return false;
        }
        __nanosleep(64);
    }
}
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort) {
    return mbar_wait_limit(b, parity, abort, kWaitCycles);
}

// Tensor maps live in global memory, where the host rewrites them between launches
// (each call uploads its descriptors into a reused workspace): the issuing thread
// orders its tensor-map reads after those generic-proxy writes, then warms the
// tensor-map cache.
__device__ __forceinline__ void tmap_acquire(const void* tm) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(tm))
                 : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(tm)) : "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(sa(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(sa(bar))
        : "memory");
}

// FP32 -> TF32 (10 explicit mantissa bits) rounded to nearest, ties away from zero,
// on the bit pattern: adding half a TF32 ulp (bit 12) to the magnitude carries into
// bit 13 exactly when the 13 dropped bits are at least half an ulp, and a carry out of
// the mantissa raises the exponent as the rounding requires.  For every finite input
// this is the value cvt.rna.tf32.f32 returns (checked over all 2^32 patterns on the
// GPU); it takes two integer operations, which issue faster than the conversion.
// NaN payloads are not preserved.
__device__ __forceinline__ uint32_t tf32_rn(float x) { return (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u; }

// K-major, 128-byte-swizzled shared-memory matrix descriptor (tcgen05):
// start address >> 4 in [0,14), leading-dim offset (unused for this layout) = 1,
// stride-dim offset = 1024 B (one 8-row x 128-B swizzle atom) in [32,46),
// version 1 in [46,48), layout SWIZZLE_128B (2) in [61,64).
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor for kind::tf32 with an FP32 accumulator: D format F32
// (bits 4-5 = 1), A and B TF32 (bits 7-9 = bits 10-12 = 2), both K-major (bits
// 15, 16 = 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_tf32(uint32_t m, uint32_t n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((n >> 3) << 17) | ((m >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}
// Instruction descriptor for kind::f16 with BF16 A and B (bits 7-9 = bits 10-12
// = 1) and an FP32 accumulator; otherwise as idesc_tf32.
__host__ __device__ constexpr uint32_t idesc_bf16(uint32_t m, uint32_t n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((m >> 4) << 24);
}

// Instruction descriptor for kind::f16 with FP16 A and B (bits 7-9 = bits 10-12 = 0)
// and an FP32 accumulator; otherwise as idesc_tf32.
__host__ __device__ constexpr uint32_t idesc_f16(uint32_t m, uint32_t n) {
    return (1u << 4) | ((n >> 3) << 17) | ((m >> 4) << 24);
}

// One K = 16 step of kind::f16 (both operands BF16 or both FP16, as the instruction
// descriptor says) with FP32 accumulation.
__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Two FP32 values rounded to nearest-even FP16 and packed, `first` in the low half.
__device__ __forceinline__ uint32_t f16x2_rn(float first, float second) {
    uint32_t r;
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(second), "f"(first));
    return r;
}
// The two FP16 halves of a packed pair back in FP32 (exact).
__device__ __forceinline__ float2 f16x2_to_f32(uint32_t h) {
    float lo, hi;
    asm("{\n\t.reg .f16 a, b;\n\tmov.b32 {a, b}, %2;\n\tcvt.f32.f16 %0, a;\n\tcvt.f32.f16 %1, b;\n\t}" : "=f"(lo), "=f"(hi) : "r"(h));
    return make_float2(lo, hi);
}
// x (|x| <= 2^15) as an FP16 pair hi + lo: hi = rn(x), lo = rn(x - hi), for two values
// at once, packed as for f16x2_rn.
__device__ __forceinline__ void split_f16x2(float a, float b, uint32_t& hi, uint32_t& lo) {
    hi = f16x2_rn(a, b);
    const float2 h = f16x2_to_f32(hi);
    lo = f16x2_rn(a - h.x, b - h.y);
}

// Two FP32 values rounded to nearest-even BF16 and packed, `first` in the low half
// (the lower address in a K-major row).
__device__ __forceinline__ uint32_t bf16x2_rn(float first, float second) {
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(second), "f"(first));
    return r;
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(sa(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// byte offset of 16-byte chunk c of row r in a 128-byte-swizzled tile (1024-B aligned)
__device__ __forceinline__ uint32_t swz(int r, int c) { return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4)); }

}  // namespace tc
}  // namespace fm

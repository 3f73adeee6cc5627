// fm_internal.cuh -- shared device/host definitions of the CUDA path (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fastmusic.h"

namespace fm {

constexpr int kLMax = 48;      // largest sketch size l handled by the small solver
constexpr int kMMax = 1024;    // largest array size M (scan keeps e^{j pi 64 m1 q}, m1 < 16, in registers)
constexpr int kKPadMax = 32;   // largest padded K in the scan

// Per-frame descriptor in device memory.  All pointers are device pointers.
struct FrameDesc {
    const float2* X;   // M x T, leading dim ldx
    int64_t ldx;
    const float2* Xin; // caller's X when X is a repacked copy (rows of T, even ldx), else null
    int64_t ldx_in;
    int M, T, K, l, t, method, L, ncols;  // ncols = columns of U_s used by the scan
    int kpad;          // padded column count of Us (multiple of 4)
    int prec;          // fm_precision of the covariance and scan GEMMs
    int refine;        // 1: one more power step C = X (X^H V) / T in FP32 before the final solve
    int scan_tc;       // 1: scanned by the tensor-core kernel (then main lobes by the fixup scan)
    int sketch_tc;     // 1: the tensor-core sketch is prepared for this frame (Bsk, tensor maps)
    int sweep_cap;     // Jacobi sweeps allowed in the l x l eigensolves (0: the solver's own cap)
    int bsk_orth_nc;   // > 0: the power-step orthonormalisation (clusters of this many CTAs)
                       // writes the B rows of the tensor-core sketch passes >= 1 itself
    float2* R;         // M x M
    float2* C;         // M x l  sketch
    float2* V;         // M x l  basis (power steps) / Q
    float2* Us;        // M x kpad (zero-padded)
    float2* Y;         // T x l  X^H V of the refinement step (refine only)
    float* Bsk;        // B rows of the tensor-core sketch (sketch_tc only): 2 l_pad x 2M, or
                       // 2 l_pad x sketch_split_rowlen(M) for a split pass
    int* idx;          // l sampled indices
    float2* qtab;      // L entries (q_hi, q_lo): q = 2 d_wl sin(theta_i), split for exact m*q_hi
    const float2* pos; // M element positions (x_hi, x_lo) in wavelengths, or null for a uniform array
    float* P;          // L
    float* Pdb;        // L (nullable)
    int* peak_idx;     // K
    float* peak_deg;   // K
    int* n_peaks;      // 1
    int* status;       // 1 (nullable)
    int* fix_list;     // L: angles the tensor-core scan leaves to the main-lobe recompute (scan_tc only)
    int* fix_count;    // 1: entries of fix_list
    uint64_t seed, frame_id;
    double theta0, step, d_wl;
};

// One CTA of the tensor-core covariance: the stages [s0, s1) (16 snapshots each) of the
// 128 x 128 output tile (ti, tj), ti <= tj, of frame `frame`.  split < 0: the item is the
// whole tile.  split >= 0: part k of the nparts items that share the tile along T; each
// writes its partial tile to slot first + k of the partial workspace, and the last one
// to finish (counter `split`) adds slots first .. first + nparts - 1 in order and writes R.
struct CovItem {
    int frame;
    int ti, tj;
    int s0, s1;
    int split;
    int first, k, nparts;
};

// One distinct angle grid: its (q_hi, q_lo) table is shared by every frame using it.
struct GridDesc {
    double theta0, step, d_wl;
    int L, pad_;
    float2* qtab;
};

// ---------------------------------------------------------------- complex ----
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// conj(a) * b
__host__ __device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}
// acc += a * b
__device__ __forceinline__ void cfma(float2& acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
}
// acc += conj(a) * b
__device__ __forceinline__ void cfmac(float2& acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(-a.y, b.x, acc.y);
}
// acc += a * conj(b)
__device__ __forceinline__ void cfmaconj(float2& acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(a.y, b.y, acc.x);
    acc.y = fmaf(a.y, b.x, acc.y);
    acc.y = fmaf(-a.x, b.y, acc.y);
}
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ float cabs2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }

// ------------------------------------------------------------ Philox4x32-10 --
// Salmon, Moraes, Dror, Shaw, SC'11.  Round: (c0..c3) -> (hi(B c2)^c1^k0, lo(B c2),
// hi(A c0)^c3^k1, lo(A c0)), A = 0xD2511F53, B = 0xCD9E8D57; key += (0x9E3779B9,
// 0xBB67AE85) between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t lo_a = 0xD2511F53u * c.x, hi_a = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo_b = 0xCD9E8D57u * c.z, hi_b = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi_b ^ c.y ^ k.x, lo_b, hi_a ^ c.w ^ k.y, lo_a);
    }
    return c;
}

// Entry (m, j) of the Gaussian test matrix of frame `frame_id` (see fastmusic.h).
__device__ __forceinline__ float2 gaussian_entry(uint64_t seed, uint64_t frame_id, int m, int j) {
    const uint4 x = philox4x32_10(make_uint4((uint32_t)j, (uint32_t)m, (uint32_t)frame_id,
                                             (uint32_t)(frame_id >> 32)),
                                  make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    // ln u1 with u1 = (x0+1)/2^32, evaluated so that it stays relatively accurate
    // near u1 = 1: there u1 = 1 - v/2^32 with v = 2^32-1-x0 exact, and log1p is used.
    float lnu1;
    if (x.x >= 0x80000000u)
        lnu1 = log1pf(-(float)(0xFFFFFFFFu - x.x) * 2.3283064365386963e-10f);
    else
        lnu1 = logf((float)(x.x + 1u) * 2.3283064365386963e-10f);
    const float u2 = (float)x.y * 2.3283064365386963e-10f;  // x1 / 2^32
    const float r = sqrtf(-2.0f * lnu1);
    float s, c;
    sincospif(2.0f * u2, &s, &c);
    return make_float2(r * c, r * s);
}

// Sorted l-subset of {0..M-1} (partial Fisher-Yates), computed by ONE thread.
// perm: scratch of M ints.
__device__ inline void sample_indices_serial(uint64_t seed, uint64_t frame_id, int M, int l, int* perm,
                                             int* out) {
    for (int m = 0; m < M; ++m) perm[m] = m;
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    for (int i = 0; i < l; ++i) {
        const uint4 x = philox4x32_10(
            make_uint4((uint32_t)i, 0xFFFFFFFFu, (uint32_t)frame_id, (uint32_t)(frame_id >> 32)), key);
        const int j = i + (int)(((uint64_t)x.x * (uint64_t)(M - i)) >> 32);
        const int tmp = perm[i];
        perm[i] = perm[j];
        perm[j] = tmp;
    }
    for (int i = 0; i < l; ++i) out[i] = perm[i];
    for (int i = 1; i < l; ++i) {
        const int v = out[i];
        int k = i - 1;
        while (k >= 0 && out[k] > v) {
            out[k + 1] = out[k];
            --k;
        }
        out[k + 1] = v;
    }
}

// e^{j pi m q} for q = q_hi + q_lo, q_hi a multiple of 2^-11 (|q| <= 2) and m < 2^11:
// m*q_hi is exact in FP32 and is reduced mod 2 without error, m*q_lo is added
// after the reduction, then one sincospif.
__device__ __forceinline__ float2 steer_exact(int m, float qh, float ql) {
    const float x = (float)m * qh;               // exact
    const float r = x - 2.0f * rintf(0.5f * x);  // exact, in [-1, 1]
    const float ph = fmaf((float)m, ql, r);
    float s, c;
    sincospif(ph, &s, &c);
    return make_float2(c, s);
}

// e^{j pi x q} for an element at x = x_hi + x_lo wavelengths (x_hi with at most 11
// significant bits) and q = q_hi + q_lo = 2 sin(theta) (q_hi a multiple of 2^-11,
// |q| <= 2): x_hi*q_hi has at most 23 significant bits, so it is exact in FP32 and is
// reduced mod 2 without error; the small terms x_hi*q_lo + x_lo*q are added after the
// reduction.  For x = m (x_lo = 0) this is steer_exact(m, q_hi, q_lo) bit for bit.
__device__ __forceinline__ float2 steer_pos(float2 x, float qh, float ql) {
    const float p = x.x * qh;                    // exact
    const float r = p - 2.0f * rintf(0.5f * p);  // exact, in [-1, 1]
    const float ph = fmaf(x.x, ql, fmaf(x.y, qh + ql, r));
    float s, c;
    sincospif(ph, &s, &c);
    return make_float2(c, s);
}

// Per-frame status bits.
__device__ __forceinline__ void set_status(int* status, int code) {
    if (status) atomicOr(status, 1 << code);
}

// Sketch products on the tensor cores (sketch_tc.cu, for frames prepared for it): every
// product R V (sampling has none at pass 0).  Every product of an FP32 frame takes three
// TF32 MMAs per FP32 product (sketch_split): the Nystrom core of Alg. 2 is built from the
// last V = orth(C), so an earlier product rounded to TF32 moves the result itself (by
// up to 3e-5 in the projector at M = 512), not only the path to it.  TF32 / BF16 frames
// take one MMA per product.
__host__ __device__ inline bool sketch_on_tc(int method, int pass) { return pass > 0 || method == FM_RAND_PROJECTION; }
__host__ __device__ inline bool sketch_split(int prec, int t, int pass) {
    (void)t;
    (void)pass;
    return prec == FM_PREC_FP32;
}
__host__ __device__ inline int sketch_tc_lpad(int l) { return (l + 7) / 8 * 8; }
// Floats per B row of the split layout: ceil(2M / 16) chunks of [hi 16 | lo 16].
__host__ __device__ inline int64_t sketch_split_rowlen(int M) { return 32 * (int64_t)((2 * M + 15) / 16); }
// Antennas of the tensor-core scan's B rows (a multiple of the 16 antennas of an FP32-mode
// stage; the TF32 and BF16 stages take 8).
__host__ __device__ inline int scan_tc_mp(int M) { return (M + 15) / 16 * 16; }

// One device -> host output copy of fm_run_host (dst: a host address the device can write).
struct CopyEntry {
    const void* src;
    void* dst;
    int64_t bytes;
};

// ---------------------------------------------------------- launch wrappers --
// Kernel launches issued by the calling host thread (every launch site bumps it),
// so the host side can report exactly how many kernels a call launched.
extern thread_local uint64_t g_kernel_launches;
inline void count_launch() { ++g_kernel_launches; }

// Programmatic dependent launch along a call's chain of kernels.  Every chain kernel
// starts with pdl_enter(): it waits until the previous kernel of the stream has
// completed and its writes are visible, so no data is read early, while the launch of
// this grid itself already overlapped the previous grid's exit (each CTA's exit is its
// trigger).  Launched without the attribute (or first in the stream) the wait returns
// at once.  An explicit trigger at CTA entry was measured slower (0.919 vs 0.839 ms per
// bench step): the next grids' CTAs were placed on the SMs the previous grid's last
// wave left free, unevenly for their own run.
__device__ __forceinline__ void pdl_enter() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Launch of a chain kernel with programmatic stream serialization (the kernel calls
// pdl_enter() before touching anything an earlier kernel wrote).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Implemented in the .cu files; each returns cudaGetLastError() after launching.
// counters (nullable): n_counters ints cleared with the status words (the covariance's
// split-tile counters, so that a run after an aborted one starts from zero)
cudaError_t launch_grid_table(const GridDesc* g, int n_grids, int max_L, const FrameDesc* d, int n_frames,
                              int* counters, int n_counters, cudaStream_t s);
cudaError_t launch_covariance_tc(const FrameDesc* d, const void* tmaps, const CovItem* items, int n_items,
                                 float2* partials, int* counters, cudaStream_t s);
constexpr int kCovTile = 128;  // complex rows per side of a covariance output tile
size_t cov_tc_smem_bytes();
cudaError_t launch_scan_tc(const FrameDesc* d, int n_frames, int M, int ncols, int L, int prec, bool pos, float* bprep,
                           const void* tmB, cudaStream_t s);
int scan_tc_ncp(int ncols);
cudaError_t launch_covariance(const FrameDesc* d, int n_frames, int max_M, cudaStream_t s);
cudaError_t launch_repack(const FrameDesc* d, int n_frames, int max_M, int max_T, cudaStream_t s);
cudaError_t launch_sketch(const FrameDesc* d, int n_frames, int max_M, int max_l, int pass, bool any_gather,
                          bool any_omega, bool any_dense, cudaStream_t s);
cudaError_t launch_orth(const FrameDesc* d, int n_frames, int max_M, int max_l, int pass, cudaStream_t s);
cudaError_t launch_final(const FrameDesc* d, int n_frames, int max_M, int max_l, cudaStream_t s);
cudaError_t launch_refine(const FrameDesc* d, int n_frames, int max_M, int max_T, cudaStream_t s);
cudaError_t launch_wait_timeout(int* status, long long limit_cycles, cudaStream_t s);
cudaError_t launch_scatter(const CopyEntry* tab, int n, cudaStream_t s);
// prep: launch the B-row preparation (false when the orthonormalisation before this pass
// wrote every frame's B rows)
cudaError_t launch_sketch_tc(const FrameDesc* d, int n_frames, int max_M, int max_l, int pass, bool any_plain,
                             bool any_split, const void* tmA, const void* tmB, const void* tmA_split,
                             const void* tmB_split, cudaStream_t s, bool prep = true);
// Cluster size of the l x l kernels for a launch over n_frames frames (small.cu).
int orth_cluster_size(int max_M, int max_l, int n_frames);
// Whether a frame's rows split into whole 8-entry chunks of the split B layout over nc
// CTAs of ceil(M / nc) rows each (then each CTA writes the B rows of its own rows).
__host__ __device__ inline bool brows_by_cluster(int M, int nc) { return nc == 1 || ((M + nc - 1) / nc) % 8 == 0; }
size_t sketch_tc_smem_bytes(int max_l, bool split);
// smem_elems: the largest M * (scan_row_stride(kpad, KP) + (positions ? 1 : 0)) over the
// frames, KP = scan_kp_class(the launch's largest kpad) (float2 elements of shared memory
// per CTA: U_s rows and the element positions)
cudaError_t launch_scan(const FrameDesc* d, int n_frames, int max_L, int max_M, int max_kpad, size_t smem_elems,
                        cudaStream_t s);
cudaError_t launch_scan_fixup(const FrameDesc* d, int n_frames, int max_L, int max_M, int max_kpad, size_t smem_elems,
                              cudaStream_t s);
__host__ __device__ inline int scan_kp_class(int max_kpad) {
    return max_kpad <= 4 ? 4 : (max_kpad <= 8 ? 8 : (max_kpad <= 16 ? 16 : 32));
}
// Row stride (elements) of U_s in the CUDA-core scan's shared memory for a frame of kpad
// columns in a launch of accumulator width KP.
__host__ __device__ inline int scan_row_stride(int kpad, int KP) { return KP == 32 ? ((kpad + 3) & ~3) : KP; }
inline size_t scan_smem_elems(int M, int kpad, bool pos, int KP) {
    return (size_t)M * (size_t)(scan_row_stride(kpad, KP) + (pos ? 1 : 0));
}
cudaError_t launch_peaks(const FrameDesc* d, int n_frames, int max_K, int max_L, cudaStream_t s);
cudaError_t launch_test_matrix(uint64_t seed, uint64_t frame_id, int M, int l, float2* out, cudaStream_t s);
cudaError_t launch_sample_indices(uint64_t seed, uint64_t frame_id, int M, int l, int* out, cudaStream_t s);
size_t small_smem_bytes(int max_M, int l);

}  // namespace fm

// scan.cu -- MUSIC pseudo-spectrum on the angle grid (Eq. 5 / Eq. 10):
//   P(theta_i) = 1 / (||a(theta_i)||^2 - ||U_s^H a(theta_i)||^2),
//   a_m(theta) = exp(j pi m q),  q = 2 d_wl sin(theta),  ||a||^2 = M
// for a uniform array; for explicit element positions x_m (wavelengths)
// a_m(theta) = exp(j pi x_m q) with q = 2 sin(theta) (steer_pos, one sincospi per
// element and angle; the positions sit in shared memory beside U_s).
//
// Steering vectors are generated in registers, never stored: each thread owns
// one angle, splits m = 64 m1 + m0 and forms a_m = c_{m1} b_{m0} with
// c_{m1} = e^{j pi 64 m1 q} (kept in registers) and b_{m0} = e^{j pi m0 q}
// (one sincospi per m0).  Every phase m*q is reduced exactly: q = q_hi + q_lo
// with q_hi a multiple of 2^-11 (so m*q_hi is exact in FP32 for m < 2^11 and
// can be reduced mod 2 without error) and m*q_lo added after reduction.  The
// q split is produced once per distinct grid by grid_table_kernel in FP64.
// U_s (M x kpad) sits in shared memory and is read as warp-wide broadcasts.
#include <float.h>

#include "fm_internal.cuh"

namespace fm {

thread_local uint64_t g_kernel_launches = 0;

namespace {

constexpr int kThreads = 256;

// blockIdx.y < n_grids: fill the (q_hi, q_lo) table of grid blockIdx.y;
// blockIdx.y == n_grids: clear the per-frame status words and the covariance's
// split-tile counters (first kernel of a run).
__global__ void grid_table_kernel(const GridDesc* __restrict__ grids, int n_grids, const FrameDesc* __restrict__ descs,
                                  int n_frames, int* __restrict__ counters, int n_counters) {
    pdl_enter();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if ((int)blockIdx.y == n_grids) {
        if (descs && i < n_frames && descs[i].status) *descs[i].status = 0;
        if (descs && i < n_frames && descs[i].fix_count) *descs[i].fix_count = 0;
        if (counters && i < n_counters) counters[i] = 0;
        return;
    }
    const GridDesc g = grids[blockIdx.y];
    if (i >= g.L) return;
    const double th = (g.theta0 + (double)i * g.step) * (3.14159265358979323846 / 180.0);
    const double q = 2.0 * g.d_wl * sin(th);
    const double qh = rint(q * 2048.0) / 2048.0;
    g.qtab[i] = make_float2((float)qh, (float)(q - qh));
}

// c_k += sum over m = 64 b + m0 (m0 = m0_begin, m0_begin + m0_stride, ... < min(64, M))
// of conj(U_s[m][k]) a_m(theta), with U_s in shared memory in rows of kp4 elements,
// zero-padded: kp4 = KP for KP <= 16 (a compile-time stride), and for KP = 32 the
// column count rounded up to 4, so that M = 1024 frames with up to 24 columns fit;
// accumulators past kp4 stay 0.
template <int KP, int NB>
__device__ __forceinline__ void accumulate_angle(const float2* __restrict__ Usm, int kp4, int M, float2 qq,
                                                 int m0_begin, int m0_stride, float2 (&acc)[KP]) {
    const int nb = (M + 63) / 64;
    float2 cb[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) cb[b] = (b < nb) ? steer_exact(64 * b, qq.x, qq.y) : make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < KP; ++k) acc[k] = make_float2(0.f, 0.f);
    const int m0_end = min(64, M);
    for (int m0 = m0_begin; m0 < m0_end; m0 += m0_stride) {
        const float2 bm = steer_exact(m0, qq.x, qq.y);
        float2 part[KP];
#pragma unroll
        for (int k = 0; k < KP; ++k) part[k] = make_float2(0.f, 0.f);
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int m = 64 * b + m0;
            if (b < nb && m < M) {
                const float2 a = cmul(cb[b], bm);
                const float4* urow = reinterpret_cast<const float4*>(Usm + m * kp4);
#pragma unroll
                for (int k2 = 0; k2 < KP / 2; ++k2) {
                    if (KP == 32 && 2 * k2 >= kp4) break;
                    const float4 u = urow[k2];
                    cfmac(part[2 * k2], make_float2(u.x, u.y), a);
                    cfmac(part[2 * k2 + 1], make_float2(u.z, u.w), a);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < KP; ++k) acc[k] = cadd(acc[k], part[k]);
    }
}

// The same sum for an array with explicit element positions (in shared memory, pos):
// one steer_pos per element; m runs over the residue class m0_begin mod m0_stride of
// each 64-element block, partial sums per block (two-level sum, as above).
template <int KP, int NB>
__device__ __forceinline__ void accumulate_angle_pos(const float2* __restrict__ Usm, int kp4,
                                                     const float2* __restrict__ pos, int M, float2 qq, int m0_begin,
                                                     int m0_stride, float2 (&acc)[KP]) {
#pragma unroll
    for (int k = 0; k < KP; ++k) acc[k] = make_float2(0.f, 0.f);
    const int nb = (M + 63) / 64;
    for (int b = 0; b < nb; ++b) {
        float2 part[KP];
#pragma unroll
        for (int k = 0; k < KP; ++k) part[k] = make_float2(0.f, 0.f);
        const int m_end = min(64 * b + 64, M);
        for (int m = 64 * b + m0_begin; m < m_end; m += m0_stride) {
            const float2 a = steer_pos(pos[m], qq.x, qq.y);
            const float4* urow = reinterpret_cast<const float4*>(Usm + m * kp4);
#pragma unroll
            for (int k2 = 0; k2 < KP / 2; ++k2) {
                if (KP == 32 && 2 * k2 >= kp4) break;
                const float4 u = urow[k2];
                cfmac(part[2 * k2], make_float2(u.x, u.y), a);
                cfmac(part[2 * k2 + 1], make_float2(u.z, u.w), a);
            }
        }
#pragma unroll
        for (int k = 0; k < KP; ++k) acc[k] = cadd(acc[k], part[k]);
    }
}

template <int KP>
__device__ __forceinline__ void store_spectrum(const FrameDesc* dp, int i, int M, const float2 (&acc)[KP]) {
    float cn = 0.f;
#pragma unroll
    for (int k = 0; k < KP; ++k) cn += cabs2(acc[k]);
    const float den = (float)M - cn;
    const float P = (den > 0.f) ? 1.0f / den : INFINITY;
    dp->P[i] = P;
    if (dp->Pdb) dp->Pdb[i] = 10.0f * log10f(fminf(P, FLT_MAX));
}

// FIXUP = false: one angle per thread over the whole grid.
// FIXUP = true: runs after the tensor-core scan and recomputes only the angles
// where ||U_s^H a||^2 = M - 1/P exceeds 4 ncols (main lobes; about ncols for an
// angle away from every source).  The tensor-core accumulator's error grows like
// u M ||U_s^H a||^2 and is biased, while the sums here stay far below that, so
// near a peak, where M - ||U_s^H a||^2 cancels, the CUDA-core value is kept.
// The tensor-core scan's epilogue lists those angles per frame (fix_list); CTA x of
// the fix_ctas(KP) of a frame takes chunks x, x + fix_ctas, ... of fix_chunk(KP) entries (one
// U_s load serves them; a frame with a short list leaves the other CTAs idle).  Each
// angle is shared by fix_groups(KP) warps, warp g taking the
// m0 residue class g (all lanes of a warp read the same U_s row: a shared-memory
// broadcast), and the partial c_k are summed in shared memory in a fixed order, so
// an angle's value does not depend on where it sits in the list.
__host__ __device__ constexpr int fix_groups(int kp) { return kp <= 8 ? 8 : (kp == 16 ? 4 : 2); }
// one round of angles per chunk (32 angles for KP <= 8), chunks spread over the CTAs so
// that one pass of a frame's CTAs covers 512 list entries
__host__ __device__ constexpr int fix_chunk(int kp) { return kThreads / 32 / fix_groups(kp) * 32; }
__host__ __device__ constexpr int fix_ctas(int kp) { return 512 / fix_chunk(kp); }

// Usm (M x kp4, zero-padded columns) <- U_s (M x kp): float4 copies issued four at a
// time when the layouts agree, else element by element.
__device__ __forceinline__ void load_us(const float2* __restrict__ Us, float2* Usm, int M, int kp, int kp4) {
    if (kp == kp4 && (reinterpret_cast<uintptr_t>(Us) & 15) == 0) {
        const int n4 = M * kp4 / 2;  // kp4 is a multiple of 4
        const float4* __restrict__ src = reinterpret_cast<const float4*>(Us);
        float4* dst = reinterpret_cast<float4*>(Usm);
        for (int e = threadIdx.x; e < n4; e += 4 * kThreads) {
            float4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (e + u * kThreads < n4) v[u] = src[e + u * kThreads];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (e + u * kThreads < n4) dst[e + u * kThreads] = v[u];
        }
        return;
    }
    for (int e = threadIdx.x; e < M * kp4; e += kThreads) {
        const int m = e / kp4, k = e % kp4;
        Usm[e] = (k < kp) ? Us[(int64_t)m * kp + k] : make_float2(0.f, 0.f);
    }
}

template <int KP, int NB, bool FIXUP>
__global__ void __launch_bounds__(kThreads) scan_kernel(const FrameDesc* __restrict__ descs) {
    pdl_enter();
    extern __shared__ float4 smem_raw[];
    float2* Usm = reinterpret_cast<float2*>(smem_raw);  // [M][kp4]
    const FrameDesc* dp = descs + blockIdx.y;
    if ((dp->scan_tc != 0) != FIXUP) return;  // the plain scan skips tensor-core frames, the fixup the others
    const int M = dp->M, L = dp->L, kp = dp->kpad, kp4 = scan_row_stride(kp, KP);
    const int i0 = blockIdx.x * kThreads;
    if (!FIXUP && i0 >= L) return;
    const float2* __restrict__ Us = dp->Us;
    constexpr int kWarps = kThreads / 32;
    __shared__ float2 s_red[FIXUP ? kThreads * 8 : 1];  // [warp][k % 8][lane]
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int n_all = 0;
    if (FIXUP) {  // chunks x, x + fix_ctas, ... of fix_chunk entries of the frame's list
        n_all = *dp->fix_count;
        if ((int)blockIdx.x * fix_chunk(KP) >= n_all) return;
    }
    load_us(Us, Usm, M, kp, kp4);
    // element positions of a non-uniform array follow U_s in shared memory
    float2* possm = Usm + (size_t)M * kp4;
    const bool has_pos = dp->pos != nullptr;
    if (has_pos)
        for (int m = threadIdx.x; m < M; m += kThreads) possm[m] = dp->pos[m];
    __syncthreads();
    float2 acc[KP];
    if (!FIXUP) {
        const int i = i0 + threadIdx.x;
        if (i >= L) return;
        if (has_pos)
            accumulate_angle_pos<KP, NB>(Usm, kp4, possm, M, dp->qtab[i], 0, 1, acc);
        else
            accumulate_angle<KP, NB>(Usm, kp4, M, dp->qtab[i], 0, 1, acc);
        store_spectrum<KP>(dp, i, M, acc);
        return;
    }
    constexpr int G = fix_groups(KP);            // warps per angle
    constexpr int kPerRound = kWarps / G * 32;   // angles per round
    const int g = w % G, grp = w / G;
    // uniform trip count: every thread reaches every __syncthreads
    constexpr int kFixChunk = fix_chunk(KP);
    for (int base = (int)blockIdx.x * kFixChunk; base < n_all; base += kFixChunk * fix_ctas(KP))
    for (int sub = 0; sub < kFixChunk; sub += kPerRound) {
        const int a = base + sub + grp * 32 + lane;
        const bool act = sub + grp * 32 + lane < kFixChunk && a < n_all;
        const int i = act ? dp->fix_list[a] : 0;
        if (act && has_pos) {
            accumulate_angle_pos<KP, NB>(Usm, kp4, possm, M, dp->qtab[i], g, G, acc);
        } else if (act) {
            accumulate_angle<KP, NB>(Usm, kp4, M, dp->qtab[i], g, G, acc);
        } else {
#pragma unroll
            for (int k = 0; k < KP; ++k) acc[k] = make_float2(0.f, 0.f);
        }
        float cn = 0.f;
#pragma unroll
        for (int kc = 0; kc < KP; kc += 8) {
#pragma unroll
            for (int k = 0; k < 8 && kc + k < KP; ++k) s_red[(w * 8 + k) * 32 + lane] = acc[kc + k];
            __syncthreads();
            if (g == 0 && act) {
#pragma unroll
                for (int k = 0; k < 8 && kc + k < KP; ++k) {
                    float2 c = make_float2(0.f, 0.f);
#pragma unroll
                    for (int h = 0; h < G; ++h) c = cadd(c, s_red[((w + h) * 8 + k) * 32 + lane]);
                    cn += cabs2(c);
                }
            }
            __syncthreads();
        }
        if (g == 0 && act) {
            const float den = (float)M - cn;
            const float P = (den > 0.f) ? 1.0f / den : INFINITY;
            dp->P[i] = P;
            if (dp->Pdb) dp->Pdb[i] = 10.0f * log10f(fminf(P, FLT_MAX));
        }
    }
}

template <int KP, int NB, bool FIXUP>
cudaError_t launch_kp(const FrameDesc* d, int n_frames, int max_L, size_t smem_elems, cudaStream_t s) {
    const size_t smem = sizeof(float2) * smem_elems;
    const size_t static_smem = FIXUP ? sizeof(float2) * kThreads * 8 : sizeof(float2);
    if (smem + static_smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(scan_kernel<KP, NB, FIXUP>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid(FIXUP ? fix_ctas(KP) : (max_L + kThreads - 1) / kThreads, n_frames);
    count_launch();
    launch_pdl(scan_kernel<KP, NB, FIXUP>, dim3(grid), dim3(kThreads), (size_t)(smem), s, d);
    return cudaGetLastError();
}

template <int NB, bool FIXUP>
cudaError_t launch_nb(const FrameDesc* d, int n_frames, int max_L, int max_kpad, size_t smem_elems, cudaStream_t s) {
    if (max_kpad <= 4) return launch_kp<4, NB, FIXUP>(d, n_frames, max_L, smem_elems, s);
    if (max_kpad <= 8) return launch_kp<8, NB, FIXUP>(d, n_frames, max_L, smem_elems, s);
    if (max_kpad <= 16) return launch_kp<16, NB, FIXUP>(d, n_frames, max_L, smem_elems, s);
    return launch_kp<32, NB, FIXUP>(d, n_frames, max_L, smem_elems, s);
}

template <bool FIXUP>
cudaError_t launch_scan_t(const FrameDesc* d, int n_frames, int max_L, int max_M, int max_kpad, size_t smem_elems,
                          cudaStream_t s) {
    if (max_M <= 128) return launch_nb<2, FIXUP>(d, n_frames, max_L, max_kpad, smem_elems, s);
    if (max_M <= 256) return launch_nb<4, FIXUP>(d, n_frames, max_L, max_kpad, smem_elems, s);
    if (max_M <= 512) return launch_nb<8, FIXUP>(d, n_frames, max_L, max_kpad, smem_elems, s);
    return launch_nb<16, FIXUP>(d, n_frames, max_L, max_kpad, smem_elems, s);
}

}  // namespace

cudaError_t launch_grid_table(const GridDesc* g, int n_grids, int max_L, const FrameDesc* d, int n_frames,
                              int* counters, int n_counters, cudaStream_t s) {
    const int gx = (max(max(max_L, d ? n_frames : 0), counters ? n_counters : 0) + 255) / 256;
    dim3 grid(gx, n_grids + 1);
    count_launch();
    launch_pdl(grid_table_kernel, dim3(grid), dim3(256), (size_t)(0), s, g, n_grids, d, n_frames, counters, n_counters);
    return cudaGetLastError();
}

cudaError_t launch_scan(const FrameDesc* d, int n_frames, int max_L, int max_M, int max_kpad, size_t smem_elems,
                        cudaStream_t s) {
    return launch_scan_t<false>(d, n_frames, max_L, max_M, max_kpad, smem_elems, s);
}

cudaError_t launch_scan_fixup(const FrameDesc* d, int n_frames, int max_L, int max_M, int max_kpad, size_t smem_elems,
                              cudaStream_t s) {
    return launch_scan_t<true>(d, n_frames, max_L, max_M, max_kpad, smem_elems, s);
}

}  // namespace fm

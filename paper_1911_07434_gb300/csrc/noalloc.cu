// noalloc.cu -- pseudo-spectrum entry point that allocates no memory.
//
// fm_spectrum keeps its frame descriptors and the per-grid steering-phase table
// in the context's workspace, which the context allocates on demand.  Some
// callers cannot allow that: a radar front end that fixes its device memory map
// at start-up and must not allocate while frames stream in, or a host framework
// that owns every device allocation itself.  fm_spectrum_noalloc runs the same
// grid-table and scan kernels with that scratch placed in the file-scope array
// below instead, so a call performs no cudaMalloc / cudaFree and needs no
// context.  The array is part of the loaded module: every GPU that loads this
// library holds it (kNoAllocScratchBytes) until the process exits.
#include <cmath>

#include "fm_internal.cuh"

namespace {

constexpr int kNoAllocMaxFrames = 64;   // frames per call
constexpr int kNoAllocMaxL = 65536;     // grid points per call
constexpr size_t kDescBytes = sizeof(fm::FrameDesc) * kNoAllocMaxFrames;
constexpr size_t kGridOff = (kDescBytes + 255) & ~size_t(255);
constexpr size_t kTabOff = kGridOff + 256;
constexpr size_t kNoAllocScratchBytes = kTabOff + sizeof(float2) * kNoAllocMaxL;  // ~524 KB

static __device__ __align__(256) unsigned char g_spectrum_scratch[kNoAllocScratchBytes];

// Device address of the scratch array on the current device.  The host-side name
// g_spectrum_scratch is only a stand-in for it; the lookup is cheap, so every call
// makes it afresh and a device reset or a new primary context between calls never
// leaves a stale address behind.
fm_status scratch_on_current_device(char** out) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_spectrum_scratch) != cudaSuccess || p == nullptr) return FM_ERR_CUDA;
    *out = static_cast<char*>(p);
    return FM_OK;
}

}  // namespace

extern "C" fm_status fm_spectrum_noalloc(const void* U, int n_frames, int M, int ncols, double d_wl,
                                         const fm_grid* grid, float* P, fm_stream stream) {
    if (!U || !grid || !P || n_frames < 1 || M < 1 || M > fm::kMMax || ncols < 1 || ncols > fm::kKPadMax ||
        (size_t)M * (size_t)((ncols + 3) / 4 * 4) > 24576 || grid->L < 1 || !(d_wl >= 0.0 && d_wl <= 1.0) ||
        !std::isfinite(grid->theta0_deg) || !std::isfinite(grid->step_deg))
        return FM_ERR_INVALID_ARG;
    if (n_frames > kNoAllocMaxFrames || grid->L > kNoAllocMaxL) return FM_ERR_INVALID_ARG;  // beyond the array
    char* scratch = nullptr;
    fm_status st = scratch_on_current_device(&scratch);
    if (st != FM_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const double d = d_wl > 0.0 ? d_wl : 0.5;

    // descriptors are built on the host stack and copied into the array
    struct {
        fm::FrameDesc f[kNoAllocMaxFrames];
    } hd;
    fm::GridDesc g{};
    g.theta0 = grid->theta0_deg;
    g.step = grid->step_deg;
    g.d_wl = d;
    g.L = grid->L;
    g.qtab = reinterpret_cast<float2*>(scratch + kTabOff);
    for (int b = 0; b < n_frames; ++b) {
        fm::FrameDesc fd{};
        fd.M = M;
        fd.L = grid->L;
        fd.ncols = fd.kpad = ncols;
        fd.Us = const_cast<float2*>(static_cast<const float2*>(U)) + (int64_t)b * M * ncols;
        fd.P = P + (int64_t)b * grid->L;
        fd.qtab = g.qtab;
        fd.theta0 = grid->theta0_deg;
        fd.step = grid->step_deg;
        fd.d_wl = d;
        hd.f[b] = fd;
    }
    // pageable source: the copy has left the host buffers when cudaMemcpyAsync returns
    cudaError_t e = cudaMemcpyAsync(scratch, hd.f, sizeof(fm::FrameDesc) * n_frames, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(scratch + kGridOff, &g, sizeof(g), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return FM_ERR_CUDA;
    const fm::FrameDesc* dd = reinterpret_cast<const fm::FrameDesc*>(scratch);
    const fm::GridDesc* dg = reinterpret_cast<const fm::GridDesc*>(scratch + kGridOff);
    e = fm::launch_grid_table(dg, 1, grid->L, nullptr, 0, nullptr, 0, s);
    if (e == cudaSuccess) e = fm::launch_scan(dd, n_frames, grid->L, M, ncols, fm::scan_smem_elems(M, ncols, false, fm::scan_kp_class(ncols)), s);
    return e == cudaSuccess ? FM_OK : FM_ERR_CUDA;
}

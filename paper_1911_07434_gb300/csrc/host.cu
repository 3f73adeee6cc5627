// host.cu -- C ABI of the library: context, validation, workspace planning,
// launch sequencing, per-stage timing and the continuous-batching server.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cstdarg>
#include <cstddef>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "fm_internal.cuh"

using fm::FrameDesc;
using fm::GridDesc;

// The struct layouts the ctypes binding mirrors (LP64).
static_assert(sizeof(fm_array) == 24 && sizeof(fm_grid) == 24 && sizeof(fm_params) == 40, "ABI struct size");
static_assert(offsetof(fm_frame, arr) == 24 && offsetof(fm_frame, grid) == 48 && offsetof(fm_frame, p) == 72 &&
                  sizeof(fm_frame) == 168,
              "fm_frame layout");

namespace {

constexpr size_t kAlign = 256;
inline size_t aup(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

enum Stage { kStGrid = 0, kStCov, kStSketch, kStOrth, kStFinal, kStScan, kStPeaks, kStRefine };
// NVTX range names of the stages (visible in a timeline profiler; no cost without one)
const char* const kStageName[FM_N_STAGES] = {"fm grid",  "fm covariance", "fm sketch", "fm orth",
                                              "fm final", "fm scan",       "fm peaks",  "fm refine"};

struct TimedEvent {
    int stage;
    cudaEvent_t a, b;
};

struct ServeReq;

}  // namespace

struct fm_ctx {
    int device = 0;
    size_t budget = 0;
    char* arena = nullptr;
    size_t arena_bytes = 0;
    // descriptor staging: a ring of pinned buffers, each reusable once the upload that
    // read it has run, so the host may prepare calls a few steps ahead of the GPU
    static constexpr int kStaging = 4;
    char* pinned[kStaging] = {};
    size_t pinned_bytes[kStaging] = {};
    cudaEvent_t staging_done[kStaging] = {};
    bool staging_pending[kStaging] = {};
    int staging_slot = 0;
    std::string err;
    unsigned timing = 0;  // bit s: stage s is bracketed by events
    std::vector<TimedEvent> pending;
    std::vector<cudaEvent_t> pool;
    double stage_ms[FM_N_STAGES] = {};
    int stage_n[FM_N_STAGES] = {};
    uint64_t launches = 0;
    int cov_path = FM_COV_AUTO;
    int last_cov_path = 0;
    int scan_path = FM_COV_AUTO;
    int last_scan_path = 0;
    int sketch_path = FM_COV_AUTO;
    int last_sketch_path = 0;
    int sweep_cap = 0;  // Jacobi sweeps allowed in the l x l eigensolves (0: the solver's own cap)
    // serving state
    struct Slot;
    std::vector<Slot*> slots;
    struct Queued {
        uint64_t ticket;
        fm_frame frame;
        size_t need;  // the frame's own workspace without split covariance tiles
    };
    std::deque<Queued> queue;
    std::map<uint64_t, int> done;  // ticket -> 1 when complete
    uint64_t next_ticket = 1;
    uint64_t serve_launches = 0;
    // set on a serving slot's private context: the arena grows with stream-ordered
    // free/alloc on that slot's stream, which other slots' work never waits for
    cudaStream_t arena_stream = nullptr;
    // fm_run_host: copy and compute streams, two device staging slots
    struct HostSlot {
        char* buf = nullptr;
        size_t bytes = 0;
        cudaEvent_t h2d = nullptr, comp = nullptr, d2h = nullptr;
        bool used = false;
        fm::CopyEntry* tab = nullptr;  // pinned: the output copies of the slot's call
        size_t tab_cap = 0;
    };
    int host_direct = -1;  // the device writes host memory through its host address (-1: not yet asked)
    HostSlot hslot[2];
    int hnext = 0;
    cudaStream_t s_h2d = nullptr, s_comp = nullptr, s_d2h = nullptr;
    // U_s of the frames of the most recent fm_run: (workspace offset, M, ncols)
    std::vector<std::tuple<size_t, int, int>> last_us;
    size_t arena_cap = 0;  // serving slot: what the budget leaves beside the other slots
};

struct fm_ctx::Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    fm_ctx* sub = nullptr;  // a private context (own arena and staging) per slot
    std::vector<uint64_t> tickets;  // the frames of the batch in flight
    bool busy = false;
};

namespace {

fm_status fail(fm_ctx* c, fm_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return s;
}

fm_status cuda_fail(fm_ctx* c, cudaError_t e, const char* what) {
    return fail(c, FM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

cudaEvent_t get_event(fm_ctx* c) {
    if (!c->pool.empty()) {
        cudaEvent_t e = c->pool.back();
        c->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Run one stage launch, bracketed by events when timing is on.
template <typename F>
fm_status stage(fm_ctx* c, int st, cudaStream_t s, F&& launch) {
    nvtxRangePushA(kStageName[st]);
    struct Pop {
        ~Pop() { nvtxRangePop(); }
    } pop;
    cudaEvent_t a = nullptr, b = nullptr;
    const bool timed = (c->timing >> st) & 1u;
    if (timed) {
        a = get_event(c);
        b = get_event(c);
        cudaEventRecord(a, s);
    }
    const uint64_t k0 = fm::g_kernel_launches;
    cudaError_t e = launch();
    c->launches += fm::g_kernel_launches - k0;
    if (e != cudaSuccess) return cuda_fail(c, e, "kernel launch");
    if (timed) {
        cudaEventRecord(b, s);
        c->pending.push_back({st, a, b});
    }
    return FM_OK;
}

fm_status set_device(fm_ctx* c) {
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    return FM_OK;
}

fm_status ensure_arena(fm_ctx* c, size_t need) {
    if (need <= c->arena_bytes) return FM_OK;
    c->last_us.clear();  // the U_s kept for fm_run_subspace go with the old workspace
    if (need > c->budget)
        return fail(c, FM_ERR_OOM_BUDGET, "workspace of %zu bytes exceeds the context budget of %zu bytes", need,
                    c->budget);
    if (c->arena_stream) {  // serving slot: free and reallocate in the slot's stream order
        if (c->arena) {
            cudaError_t e = cudaFreeAsync(c->arena, c->arena_stream);
            if (e != cudaSuccess) return cuda_fail(c, e, "cudaFreeAsync(workspace)");
            c->arena = nullptr;
            c->arena_bytes = 0;
        }
        const size_t cap = std::min(c->budget, c->arena_cap);
        if (need > cap)
            return fail(c, FM_ERR_OOM_BUDGET, "workspace of %zu bytes exceeds the %zu bytes left in the budget", need,
                        cap);
        size_t sz = std::min(cap, need + need / 4);
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&c->arena), sz, c->arena_stream);
        if (e != cudaSuccess) {
            c->arena = nullptr;
            return cuda_fail(c, e, "cudaMallocAsync(workspace)");
        }
        c->arena_bytes = sz;
        return FM_OK;
    }
    if (c->arena) {
        cudaError_t e = cudaDeviceSynchronize();  // the old arena may still be read by queued work
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaDeviceSynchronize");
        cudaFree(c->arena);
        c->arena = nullptr;
        c->arena_bytes = 0;
    }
    size_t sz = std::min(c->budget, std::max(need, need + need / 4));
    cudaError_t e = cudaMalloc(&c->arena, sz);
    if (e != cudaSuccess) {
        c->arena = nullptr;
        return cuda_fail(c, e, "cudaMalloc(workspace)");
    }
    c->arena_bytes = sz;
    return FM_OK;
}

// Pinned staging for descriptor uploads; waits for the previous upload first.
// The current slot of the staging ring, at least `need` bytes, once the upload that last
// read it has run.
fm_status staging(fm_ctx* c, size_t need, char** out) {
    const int k = c->staging_slot;
    if (c->staging_pending[k]) {
        cudaEventSynchronize(c->staging_done[k]);
        c->staging_pending[k] = false;
    }
    if (need > c->pinned_bytes[k]) {
        if (c->pinned[k]) cudaFreeHost(c->pinned[k]);
        size_t sz = std::max(need, (size_t)1 << 16);
        cudaError_t e = cudaMallocHost(&c->pinned[k], sz);
        if (e != cudaSuccess) {
            c->pinned[k] = nullptr;
            c->pinned_bytes[k] = 0;
            return cuda_fail(c, e, "cudaMallocHost(staging)");
        }
        c->pinned_bytes[k] = sz;
    }
    *out = c->pinned[k];
    return FM_OK;
}

// Copies the current staging slot (host) to dev on s and moves to the next slot.
fm_status upload(fm_ctx* c, const char* host, char* dev, size_t bytes, cudaStream_t s) {
    const int k = c->staging_slot;
    cudaError_t e = cudaMemcpyAsync(dev, host, bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemcpyAsync(descriptors)");
    if (!c->staging_done[k]) cudaEventCreateWithFlags(&c->staging_done[k], cudaEventDisableTiming);
    cudaEventRecord(c->staging_done[k], s);
    c->staging_pending[k] = true;
    c->staging_slot = (k + 1) % fm_ctx::kStaging;
    return FM_OK;
}

int ncols_of(const fm_params& p) {
    return (p.rank_restrict == p.l) ? p.l : p.K;
}

const char* check_frame(const fm_frame& f) {
    const fm_params& p = f.p;
    const int M = f.arr.M;
    if (!f.X) return "X is NULL";
    if (M < 2 || M > fm::kMMax) return "M must be in [2, 1024]";
    if (f.T < 1) return "T must be >= 1";
    if (f.ldx < f.T) return "ldx must be >= T";
    if (f.arr.pos_wl) {
        for (int m = 0; m < M; ++m)
            if (!(std::fabs(f.arr.pos_wl[m]) <= 4096.0)) return "pos_wl: positions must be finite with |x| <= 4096";
    } else if (!(f.arr.d_wl >= 0.0 && f.arr.d_wl <= 1.0)) {
        return "d_wl must be in (0, 1] (0 selects 0.5)";
    }
    if (f.grid.L < 1 || f.grid.L > 65536) return "grid L must be in [1, 65536]";
    if (!std::isfinite(f.grid.theta0_deg) || !std::isfinite(f.grid.step_deg)) return "grid is not finite";
    if (p.method != FM_RAND_SAMPLING && p.method != FM_RAND_PROJECTION) return "method must be 1 or 2";
    if (p.K < 1 || p.K > p.l) return "need 1 <= K <= l";
    if (p.l > M || p.l > fm::kLMax) return "need l <= min(M, 48)";
    if (p.t < 0 || p.t > 8) return "t must be in [0, 8]";
    if (p.prec != FM_PREC_FP32 && p.prec != FM_PREC_TF32 && p.prec != FM_PREC_BF16) return "prec must be 0, 1 or 2";
    if (p.refine != 0 && p.refine != 1) return "refine must be 0 or 1";
    if (p.rank_restrict != 0 && p.rank_restrict != p.K && p.rank_restrict != p.l) return "rank_restrict must be 0, K or l";
    const int nc = ncols_of(p);
    if (nc > fm::kKPadMax) return "columns of U_s used by the scan must be <= 32";
    if ((size_t)M * (size_t)((nc + 3) / 4 * 4) > 24576) return "M * ceil4(ncols) must be <= 24576";
    if (!f.P_out || !f.peak_idx || !f.peak_deg || !f.n_peaks) return "an output pointer is NULL";
    return nullptr;
}

// Spacing that enters the grid's phase table q = 2 d sin(theta): the ULA spacing, or
// 1 for explicit positions (the element phase is then pi x_m q = 2 pi x_m sin(theta)).
double grid_spacing(const fm_frame& f) {
    if (f.arr.pos_wl) return 1.0;
    return f.arr.d_wl > 0.0 ? f.arr.d_wl : 0.5;
}

// x = hi + lo with hi carrying at most 11 significant bits, so that hi * q_hi is exact in
// FP32 for any q_hi that is a multiple of 2^-11 with |q_hi| <= 2 (at most 23 bits).
float2 split_position(double x) {
    if (x == 0.0) return make_float2(0.f, 0.f);
    int e = 0;
    std::frexp(x, &e);  // |x| in [2^(e-1), 2^e)
    const double scale = std::ldexp(1.0, 11 - e);
    const double hi = std::nearbyint(x * scale) / scale;
    return make_float2((float)hi, (float)(x - hi));
}

// Geometry id per frame: 0 for a uniform array, k >= 1 for the k-th distinct set of
// element positions (compared element by element), in order of first appearance.
std::vector<int> geometry_ids(const fm_frame* f, int n, std::vector<const fm_frame*>* firsts = nullptr) {
    std::vector<int> id(n, 0);
    std::vector<const fm_frame*> reps;
    for (int b = 0; b < n; ++b) {
        if (!f[b].arr.pos_wl) continue;
        int k = 0;
        for (size_t r = 0; r < reps.size() && !k; ++r)
            if (reps[r]->arr.M == f[b].arr.M &&
                (reps[r]->arr.pos_wl == f[b].arr.pos_wl ||
                 std::memcmp(reps[r]->arr.pos_wl, f[b].arr.pos_wl, sizeof(double) * (size_t)f[b].arr.M) == 0))
                k = (int)r + 1;
        if (!k) {
            reps.push_back(&f[b]);
            k = (int)reps.size();
        }
        id[b] = k;
    }
    if (firsts) *firsts = reps;
    return id;
}

// SM count of the current device (152 on GB300; the fallback when no device answers,
// e.g. for host-only workspace sizing).
int current_sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
        n > 0)
        return n;
    cudaGetLastError();
    return 152;
}

// Work items of the tensor-core covariance (see cov_tc.cu).  Each 128 x 128 tile of
// the upper block triangle of every frame is one item, weighted in quarter stages (an
// off-diagonal tile issues 4 blocks per 16-snapshot stage, a diagonal tile 3), plus a
// fixed cost per CTA (prologue, first loads, epilogue: about six stages).  Items stay
// grouped by frame (the tiles of a frame run side by side and read its X from L2 once),
// frames ordered by their work, largest first, off-diagonal tiles before diagonal ones.
// A greedy simulation of that launch order on n_sm SMs (one CTA per SM) finds the tiles
// that would still run after every other SM has finished; those are split along T into
// s parts in place (s in 2..8, the s that shortens the simulated makespan most; each
// part keeps at least 4 stages).  Small batches gain most: one M = 512 frame's 10 tiles
// become 80 parts on 152 SMs.
struct CovPlan {
    std::vector<fm::CovItem> items;
    int n_split = 0, n_slots = 0;
};

// Costs in quarter stages (one quarter of an off-diagonal tile's 16-snapshot stage,
// about 420 SM cycles), measured per CTA on GB300: the prologue, the epilogue (TMEM ->
// shared -> R and its mirror at about 30 bytes per cycle) and the launch gap of a CTA;
// the partial tile a split part writes; the reduction that the last part of a tile
// split in s adds (it reads the s partials, then writes the tile).
constexpr int64_t kCovCtaCost = 64;
// At most two partial tiles per SM (39 MB of partial workspace on 152 SMs), whatever
// the batch, so that a batch's workspace is bounded by its frames' own plus this.
inline int64_t cov_max_slots(int n_sm) { return 2 * (int64_t)n_sm; }
inline size_t cov_split_cap_bytes(int n_sm) {
    return (size_t)cov_max_slots(n_sm) * (sizeof(float2) * fm::kCovTile * fm::kCovTile + sizeof(int)) + 512;
}
constexpr int64_t kCovPartCost = 24;
inline int64_t cov_reduce_cost(int s) { return 36 + 12 * (int64_t)s; }

// Greedy simulation of a launch: each item, in order, starts on the SM that frees up
// first; returns the makespan (and each item's end time).
int64_t lpt_makespan(const std::vector<int64_t>& w, int n_sm, std::vector<int64_t>* ends = nullptr) {
    std::vector<int64_t> heap(n_sm, 0);  // min-heap of SM finish times
    auto cmp = [](int64_t a, int64_t b) { return a > b; };
    int64_t mk = 0;
    if (ends) ends->resize(w.size());
    for (size_t i = 0; i < w.size(); ++i) {
        std::pop_heap(heap.begin(), heap.end(), cmp);
        const int64_t e = heap.back() + w[i];
        heap.back() = e;
        std::push_heap(heap.begin(), heap.end(), cmp);
        if (ends) (*ends)[i] = e;
        mk = std::max(mk, e);
    }
    return mk;
}

// Indices of w sorted by weight, largest first, equal weights in index order.
std::vector<int> longest_first(const std::vector<int64_t>& w) {
    std::vector<int> order(w.size());
    for (size_t i = 0; i < w.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return w[a] > w[b]; });
    return order;
}

// Second launch order, for batches of a few waves: the SMs in two lanes, one running
// the off-diagonal tiles and one the cheaper diagonal tiles, each lane list-scheduled
// in frame order, the lane sizes balancing the two makespans.  The items launch in the
// order of their planned start times (lane by lane at equal times), so the SM that
// frees up next takes the next item of its own lane.  Equal frames then reach the
// packing bound where the frame order leaves a last partial wave: 64 frames of
// M = 512 on 152 SMs give 96 SMs four off-diagonal tiles each and 56 SMs four or five
// diagonal ones (simulated makespan 1280 against 1408 quarter stages).
void order_in_lanes(std::vector<fm::CovItem>& tiles, std::vector<int64_t>& w, int n_sm) {
    std::vector<int> ia, ib;
    for (size_t i = 0; i < tiles.size(); ++i) (tiles[i].ti != tiles[i].tj ? ia : ib).push_back((int)i);
    if (ia.empty() || ib.empty() || n_sm < 2) return;
    auto lane = [&](const std::vector<int>& idx, int nsm, std::vector<int64_t>* starts) {
        std::vector<int64_t> wl(idx.size()), ends;
        for (size_t k = 0; k < idx.size(); ++k) wl[k] = w[idx[k]] + kCovCtaCost;
        const int64_t mk = lpt_makespan(wl, nsm, starts ? &ends : nullptr);
        if (starts) {
            starts->resize(idx.size());
            for (size_t k = 0; k < idx.size(); ++k) (*starts)[k] = ends[k] - wl[k];
        }
        return mk;
    };
    auto both = [&](int na) { return std::max(lane(ia, na, nullptr), lane(ib, n_sm - na, nullptr)); };
    // the smallest lane a whose makespan is at most lane b's (a's shrinks, b's grows with na)
    int lo = 1, hi = n_sm - 1;
    while (lo < hi) {
        const int mid = (lo + hi) / 2;
        if (lane(ia, mid, nullptr) <= lane(ib, n_sm - mid, nullptr))
            hi = mid;
        else
            lo = mid + 1;
    }
    int na = lo;
    if (lo > 1 && both(lo - 1) < both(lo)) na = lo - 1;
    std::vector<int64_t> sa_, sb_;
    lane(ia, na, &sa_);
    lane(ib, n_sm - na, &sb_);
    std::vector<std::tuple<int64_t, int, int>> ev;
    ev.reserve(tiles.size());
    for (size_t k = 0; k < ia.size(); ++k) ev.emplace_back(sa_[k], 0, ia[k]);
    for (size_t k = 0; k < ib.size(); ++k) ev.emplace_back(sb_[k], 1, ib[k]);
    std::sort(ev.begin(), ev.end());
    std::vector<fm::CovItem> t2;
    std::vector<int64_t> w2;
    t2.reserve(tiles.size());
    w2.reserve(tiles.size());
    for (const auto& e : ev) {
        t2.push_back(tiles[std::get<2>(e)]);
        w2.push_back(w[std::get<2>(e)]);
    }
    tiles.swap(t2);
    w.swap(w2);
}

CovPlan plan_cov_items_uncached(const fm_frame* f, int n, int n_sm, bool allow_split) {
    // frames by total tile work, largest first (ties in the caller's order)
    std::vector<int64_t> fw(n);
    for (int b = 0; b < n; ++b) {
        const int64_t nt = (f[b].arr.M + fm::kCovTile - 1) / fm::kCovTile;
        fw[b] = (int64_t)((f[b].T + 15) / 16) * (4 * nt * (nt - 1) / 2 + 3 * nt);
    }
    const std::vector<int> forder = longest_first(fw);
    std::vector<fm::CovItem> tiles;
    std::vector<int64_t> w;
    for (int b : forder) {
        const int nt = (f[b].arr.M + fm::kCovTile - 1) / fm::kCovTile;
        const int ns = (f[b].T + 15) / 16;
        for (int ti = 0; ti < nt; ++ti)
            for (int tj = ti + 1; tj < nt; ++tj) {
                tiles.push_back(fm::CovItem{b, ti, tj, 0, ns, -1, 0, 0, 1});
                w.push_back((int64_t)ns * 4);
            }
        for (int ti = 0; ti < nt; ++ti) {
            tiles.push_back(fm::CovItem{b, ti, ti, 0, ns, -1, 0, 0, 1});
            w.push_back((int64_t)ns * 3);
        }
    }
    if (n_sm > 1 && (int64_t)tiles.size() > n_sm && (int64_t)tiles.size() <= 8 * (int64_t)n_sm) {
        std::vector<fm::CovItem> t2 = tiles;
        std::vector<int64_t> w2 = w, wo1(w.size()), wo2;
        order_in_lanes(t2, w2, n_sm);
        for (size_t i = 0; i < w.size(); ++i) wo1[i] = w[i] + kCovCtaCost;
        for (int64_t x : w2) wo2.push_back(x + kCovCtaCost);
        if ((double)lpt_makespan(wo2, n_sm) < 0.99 * (double)lpt_makespan(wo1, n_sm)) {
            tiles.swap(t2);
            w.swap(w2);
        }
    }
    CovPlan plan;
    std::vector<int64_t> wo(tiles.size());
    int64_t total = 0;
    for (size_t i = 0; i < tiles.size(); ++i) total += (wo[i] = w[i] + kCovCtaCost);
    int best_s = 1;
    std::vector<int64_t> ends;
    const double late = n_sm > 0 ? 1.02 * (double)total / n_sm : 0.0;  // finishing later: split candidates
    auto is_candidate = [&](size_t i, int s) { return (double)ends[i] > late && tiles[i].s1 >= 4 * s; };
    if (allow_split && n_sm > 0 && (int64_t)tiles.size() <= 8 * (int64_t)n_sm) {
        int64_t best = lpt_makespan(wo, n_sm, &ends);
        for (int s : {2, 3, 4, 6, 8}) {
            int64_t slots = 0;
            for (size_t i = 0; i < tiles.size(); ++i) slots += is_candidate(i, s) ? s : 0;
            if (slots > cov_max_slots(n_sm)) continue;  // the partial workspace stays bounded
            std::vector<int64_t> cand;
            for (size_t i = 0; i < tiles.size(); ++i) {
                if (is_candidate(i, s))
                    for (int k = 0; k < s; ++k)
                        cand.push_back(w[i] / s + kCovCtaCost + kCovPartCost + (k == s - 1 ? cov_reduce_cost(s) : 0));
                else
                    cand.push_back(wo[i]);
            }
            const int64_t mk = lpt_makespan(cand, n_sm);
            if ((double)mk < 0.99 * (double)best) {
                best = mk;
                best_s = s;
            }
        }
    }
    // the items in launch order; the parts of a split tile take its place
    plan.items.reserve(tiles.size());
    for (size_t i = 0; i < tiles.size(); ++i) {
        const fm::CovItem t = tiles[i];
        if (best_s == 1 || !is_candidate(i, best_s)) {
            plan.items.push_back(t);
            continue;
        }
        const int ns = t.s1;
        for (int k = 0; k < best_s; ++k) {
            fm::CovItem p = t;
            p.s0 = (int)((int64_t)ns * k / best_s);
            p.s1 = (int)((int64_t)ns * (k + 1) / best_s);
            p.split = plan.n_split;
            p.first = plan.n_slots;
            p.k = k;
            p.nparts = best_s;
            plan.items.push_back(p);
        }
        ++plan.n_split;
        plan.n_slots += best_s;
    }
    return plan;
}

// The plan depends only on each frame's M and T (in the order given), the SM count and
// allow_split; a caller that repeats its batch shape (a stream of equal batches, the
// serving slots) gets the last plan of its thread back without the simulations, which
// take a few hundred microseconds of host time for a 64-frame batch.
CovPlan plan_cov_items(const fm_frame* f, int n, int n_sm, bool allow_split) {
    thread_local std::vector<int64_t> key;
    thread_local CovPlan plan;
    std::vector<int64_t> k;
    k.reserve(2 * (size_t)n + 2);
    k.push_back(n_sm);
    k.push_back(allow_split ? 1 : 0);
    for (int b = 0; b < n; ++b) {
        k.push_back(f[b].arr.M);
        k.push_back(f[b].T);
    }
    if (k != key) {
        plan = plan_cov_items_uncached(f, n, n_sm, allow_split);
        key.swap(k);
    }
    return plan;
}

struct Plan {
    size_t desc_off, tmap_off, grid_off, pos_off, upload_bytes, total;
    // tensor-core scan groups: maximal runs of consecutive frames sharing M, ncols,
    // grid and prec (fm_run orders the frames so that each group is one run)
    struct ScanGroup {
        int f0, nf, M, nc, L, prec;
        size_t bprep_off, rows, rowlen;
    };
    std::vector<ScanGroup> scan_groups;
    std::vector<size_t> R, C, V, Us, idx, Y;  // per-frame offsets (R == SIZE_MAX: caller-owned)
    std::vector<size_t> fix;   // main-lobe list (L ints) and its count of a tensor-core scan (SIZE_MAX: none)
    std::vector<size_t> Xpad;  // repacked copy of X for the tensor-core covariance (SIZE_MAX: none)
    std::vector<size_t> Bsk;   // B rows of the tensor-core sketch (SIZE_MAX: none)
    std::vector<int> grid_of;
    std::vector<GridDesc> grids;
    std::vector<size_t> qtab;
    // element positions (split as (hi, lo) floats), one table per distinct geometry,
    // uploaded with the descriptors; geom_of[b] = 0 for a uniform array
    std::vector<int> geom_of;
    std::vector<size_t> pos_tab;        // offset of geometry k's table (index k - 1)
    std::vector<float2> pos_host;       // every table back to back
    std::vector<size_t> pos_host_at;    // start of table k - 1 in pos_host
    // tensor-core covariance work items (uploaded), partial tiles and counters of split tiles
    CovPlan cov;
    size_t cov_items_off = 0, cov_part_off = 0, cov_cnt_off = 0;
};

typedef std::tuple<double, double, double, int> GridKey;

// Lays out the workspace for n frames.  need_R etc. say which buffers live in the workspace.
Plan plan_frames(const fm_frame* f, int n, bool need_R, bool need_sketch, bool need_Us, bool need_grid,
                 bool allow_split = true) {
    Plan pl;
    size_t off = 0;
    pl.desc_off = off;
    off = aup(off + sizeof(FrameDesc) * (size_t)n);
    // TMA tensor maps: per frame X (covariance); per scan group B; per frame the R and
    // B-row maps of the tensor-core sketch, one-MMA and split layouts
    pl.tmap_off = off;
    if (need_R) off = aup(off + sizeof(CUtensorMap) * (6 * (size_t)n));
    std::map<GridKey, int> gmap;
    pl.grid_of.assign(n, -1);
    if (need_grid) {
        for (int b = 0; b < n; ++b) {
            const double d = grid_spacing(f[b]);
            GridKey k(f[b].grid.theta0_deg, f[b].grid.step_deg, d, f[b].grid.L);
            auto it = gmap.find(k);
            if (it == gmap.end()) {
                const int g = (int)pl.grids.size();
                gmap[k] = g;
                GridDesc gd{};
                gd.theta0 = f[b].grid.theta0_deg;
                gd.step = f[b].grid.step_deg;
                gd.d_wl = d;
                gd.L = f[b].grid.L;
                pl.grids.push_back(gd);
                pl.grid_of[b] = g;
            } else {
                pl.grid_of[b] = it->second;
            }
        }
    }
    pl.grid_off = off;
    off = aup(off + sizeof(GridDesc) * pl.grids.size());
    pl.pos_off = off;
    pl.geom_of.assign(n, 0);
    if (need_grid) {
        std::vector<const fm_frame*> reps;
        pl.geom_of = geometry_ids(f, n, &reps);
        for (const fm_frame* r : reps) {
            pl.pos_tab.push_back(off);
            pl.pos_host_at.push_back(pl.pos_host.size());
            for (int m = 0; m < r->arr.M; ++m) pl.pos_host.push_back(split_position(r->arr.pos_wl[m]));
            off = aup(off + sizeof(float2) * (size_t)r->arr.M);
        }
    }
    if (need_R) {
        pl.cov = plan_cov_items(f, n, current_sm_count(), allow_split);
        pl.cov_items_off = off;
        off = aup(off + sizeof(fm::CovItem) * pl.cov.items.size());
    }
    pl.upload_bytes = off;
    if (need_R && pl.cov.n_split) {
        pl.cov_part_off = off;
        off = aup(off + sizeof(float2) * (size_t)fm::kCovTile * fm::kCovTile * (size_t)pl.cov.n_slots);
        pl.cov_cnt_off = off;
        off = aup(off + sizeof(int) * (size_t)pl.cov.n_split);
    }
    for (size_t g = 0; g < pl.grids.size(); ++g) {
        pl.qtab.push_back(off);
        off = aup(off + sizeof(float2) * (size_t)pl.grids[g].L);
    }
    for (int b = 0; b < n; ++b) {
        const size_t M = (size_t)f[b].arr.M, l = (size_t)f[b].p.l;
        // TMA needs a 16-byte aligned base and an even ldx: other frames get a padded copy
        const bool pad = need_R && ((reinterpret_cast<uintptr_t>(f[b].X) % 16) != 0 || (f[b].ldx % 2) != 0);
        pl.Xpad.push_back(pad ? off : SIZE_MAX);
        if (pad) off = aup(off + sizeof(float2) * M * (size_t)(f[b].T + (f[b].T & 1)));
        pl.R.push_back(need_R ? off : SIZE_MAX);
        if (need_R) off = aup(off + sizeof(float2) * M * M);
        pl.C.push_back(need_sketch ? off : SIZE_MAX);
        if (need_sketch) off = aup(off + sizeof(float2) * M * l);
        pl.V.push_back(need_sketch ? off : SIZE_MAX);
        if (need_sketch) off = aup(off + sizeof(float2) * M * l);
        pl.idx.push_back(need_sketch ? off : SIZE_MAX);
        if (need_sketch) off = aup(off + sizeof(int) * l);
        bool tcsk = false;  // some pass of this frame can run on the tensor-core sketch
        for (int pass = 0; need_R && pass <= f[b].p.t; ++pass) tcsk |= fm::sketch_on_tc(f[b].p.method, pass);
        pl.Bsk.push_back(tcsk ? off : SIZE_MAX);  // sized for the split layout (the larger)
        if (tcsk)
            off = aup(off + sizeof(float) * 2 * (size_t)fm::sketch_tc_lpad((int)l) *
                                (size_t)fm::sketch_split_rowlen((int)M));
        const bool y = need_sketch && f[b].p.refine;  // X^H V of the refinement step
        pl.Y.push_back(y ? off : SIZE_MAX);
        if (y) off = aup(off + sizeof(float2) * (size_t)f[b].T * l);
        const size_t nc = (size_t)ncols_of(f[b].p);
        pl.Us.push_back(need_Us ? off : SIZE_MAX);
        if (need_Us) off = aup(off + sizeof(float2) * M * nc);
        const bool fx = need_R && need_Us && need_grid;  // the frame may take the tensor-core scan
        pl.fix.push_back(fx ? off : SIZE_MAX);
        if (fx) off = aup(off + sizeof(int) * ((size_t)f[b].grid.L + 1));
    }
    if (need_R && need_Us && need_grid) {
        for (int b = 0; b < n;) {
            const int M0 = f[b].arr.M, nc0 = ncols_of(f[b].p), pr0 = f[b].p.prec, g0 = pl.grid_of[b];
            int e = b + 1;
            const int geo0 = pl.geom_of[b];
            while (e < n && f[e].arr.M == M0 && ncols_of(f[e].p) == nc0 && f[e].p.prec == pr0 &&
                   pl.grid_of[e] == g0 && pl.geom_of[e] == geo0)
                ++e;
            Plan::ScanGroup sg{};
            sg.f0 = b;
            sg.nf = e - b;
            sg.M = M0;
            sg.nc = nc0;
            sg.L = pl.grids[g0].L;
            sg.prec = pr0;
            const int ncp = fm::scan_tc_ncp(nc0), Mp = fm::scan_tc_mp(M0);
            sg.rows = (size_t)sg.nf * 2 * ncp;  // one B operand row pair per (frame, column of U_s)
            sg.rowlen = 4 * (size_t)Mp;
            sg.bprep_off = off;
            off = aup(off + sizeof(float) * sg.rows * sg.rowlen);
            pl.scan_groups.push_back(sg);
            b = e;
        }
    }
    pl.total = off;
    return pl;
}

FrameDesc make_desc(const fm_frame& f) {
    FrameDesc d{};
    d.X = reinterpret_cast<const float2*>(f.X);
    d.ldx = f.ldx;
    d.M = f.arr.M;
    d.T = f.T;
    d.K = f.p.K;
    d.l = f.p.l;
    d.t = f.p.t;
    d.method = f.p.method;
    d.L = f.grid.L;
    d.ncols = ncols_of(f.p);
    d.kpad = d.ncols;
    d.prec = f.p.prec;
    d.refine = f.p.refine;
    d.P = f.P_out;
    d.Pdb = f.P_db_out;
    d.peak_idx = f.peak_idx;
    d.peak_deg = f.peak_deg;
    d.n_peaks = f.n_peaks;
    d.status = f.status;
    d.seed = f.p.seed;
    d.frame_id = f.frame_id;
    d.theta0 = f.grid.theta0_deg;
    d.step = f.grid.step_deg;
    d.d_wl = grid_spacing(f);
    return d;
}

struct Maxes {
    int M = 0, l = 0, L = 0, K = 0, kpad = 0, t = 0, T = 0;
    bool any_sampling = false, any_projection = false, any_status = false, any_refine = false, any_pos = false;
    size_t scan_smem = 0;  // float2 elements of shared memory the CUDA-core scan needs
};

Maxes maxes_of(const std::vector<FrameDesc>& ds) {
    Maxes m;
    for (const FrameDesc& d : ds) {
        m.M = std::max(m.M, d.M);
        m.l = std::max(m.l, d.l);
        m.L = std::max(m.L, d.L);
        m.K = std::max(m.K, d.K);
        m.kpad = std::max(m.kpad, d.kpad);
        m.t = std::max(m.t, d.t);
        m.T = std::max(m.T, d.T);
        m.any_refine |= d.refine != 0;
        m.any_sampling |= d.method == FM_RAND_SAMPLING;
        m.any_projection |= d.method == FM_RAND_PROJECTION;
        m.any_status |= d.status != nullptr;
        m.any_pos |= d.pos != nullptr;
    }
    const int KP = fm::scan_kp_class(m.kpad);
    for (const FrameDesc& d : ds)
        m.scan_smem = std::max(m.scan_smem, fm::scan_smem_elems(d.M, d.kpad, d.pos != nullptr, KP));
    return m;
}

// ---- TMA tensor maps for the tensor-core covariance ----------------------
PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// A frame can take the tensor-core path if its rows can be described to TMA:
// 16-byte aligned base and an even leading dimension (row stride multiple of 16 B).
bool tc_eligible(const FrameDesc& d) {
    return (reinterpret_cast<uintptr_t>(d.X) % 16 == 0) && (d.ldx % 2 == 0) && d.M >= 1 && d.T >= 1 &&
           (int64_t)2 * d.T < ((int64_t)1 << 32);
}

// X viewed as an M x 2T FP32 matrix, boxes of 128 rows x 32 floats, 128-byte swizzle.
bool encode_tmap(const FrameDesc& d, CUtensorMap* out) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)(2 * (int64_t)d.T), (cuuint64_t)d.M};
    cuuint64_t strides[1] = {(cuuint64_t)(d.ldx * 8)};
    cuuint32_t box[2] = {32, 128};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float2*>(d.X), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// The tensor-core sketch: R viewed as M x 2M FP32 (boxes of 128 rows x 32 floats,
// 128-byte swizzle) and its B rows (2 l_pad x 2M FP32, one box of all 2 l_pad rows x
// 32 floats); for the split kernel, R in raw boxes of 128 rows x 16 floats (no
// swizzle) and the split B rows (2 l_pad x sketch_split_rowlen(M), boxes of 32 floats).
bool encode_sketch_tmaps(const FrameDesc& d, CUtensorMap* a, CUtensorMap* b, CUtensorMap* a2, CUtensorMap* b2) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
    if (!enc) return false;
    const int nb = 2 * fm::sketch_tc_lpad(d.l);
    cuuint64_t dims[2] = {(cuuint64_t)(2 * (int64_t)d.M), (cuuint64_t)d.M};
    cuuint64_t strides[1] = {(cuuint64_t)d.M * 8};
    cuuint32_t box[2] = {32, 128};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(a, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, d.R, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
    cuuint64_t dims_b[2] = {(cuuint64_t)(2 * (int64_t)d.M), (cuuint64_t)nb};
    cuuint32_t box_b[2] = {32, (cuuint32_t)nb};
    r = enc(b, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, d.Bsk, dims_b, strides, box_b, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
    cuuint32_t box_raw[2] = {16, 128};
    r = enc(a2, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, d.R, dims, strides, box_raw, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
    const int64_t rl = fm::sketch_split_rowlen(d.M);
    cuuint64_t dims_s[2] = {(cuuint64_t)rl, (cuuint64_t)nb};
    cuuint64_t strides_s[1] = {(cuuint64_t)rl * 4};
    r = enc(b2, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, d.Bsk, dims_s, strides_s, box_b, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// The scan's B operand (rows x rowlen FP32, rowlen = 4 Mp), boxes of 256 rows x 32 floats.
bool encode_bprep_tmap(const float* base, size_t rows, size_t rowlen, CUtensorMap* out) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)rowlen, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(rowlen * sizeof(float))};
    cuuint32_t box[2] = {32, 256};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// Decide the covariance path for these frames and, for the tensor-core path,
// encode one tensor map per frame.  Fails only if the context forces the
// tensor-core path and a frame cannot take it.
fm_status choose_cov_path(fm_ctx* c, const std::vector<FrameDesc>& ds, std::vector<CUtensorMap>& maps, bool* tc_out) {
    bool tc = (c->cov_path != FM_COV_SIMT);
    for (size_t b = 0; tc && b < ds.size(); ++b) tc = tc_eligible(ds[b]);
    if (tc) {
        maps.resize(ds.size());
        for (size_t b = 0; tc && b < ds.size(); ++b) tc = encode_tmap(ds[b], &maps[b]);
    }
    if (!tc) maps.clear();
    if (!tc && c->cov_path == FM_COV_TC)
        return fail(c, FM_ERR_INVALID_ARG, "tensor-core covariance needs 16-byte aligned X with an even ldx");
    c->last_cov_path = tc ? FM_COV_TC : FM_COV_SIMT;
    *tc_out = tc;
    return FM_OK;
}

// items / partials / counters: the tensor-core path's work items (device) and the
// workspace of its split tiles (null when no tile is split)
fm_status launch_cov(fm_ctx* c, bool tc, FrameDesc* dd, const char* tm_dev, const fm::CovItem* items, int n_items,
                     float2* partials, int* counters, int n, int max_M, cudaStream_t s) {
    if (tc)
        return stage(c, 1, s, [&] { return fm::launch_covariance_tc(dd, tm_dev, items, n_items, partials, counters, s); });
    return stage(c, 1, s, [&] { return fm::launch_covariance(dd, n, max_M, s); });
}

// Uploads descriptors (+ grids) and returns device pointers.
fm_status upload_descs(fm_ctx* c, const Plan& pl, std::vector<FrameDesc>& ds, const std::vector<CUtensorMap>& maps,
                       cudaStream_t s, FrameDesc** dd, GridDesc** dg,
                       const std::vector<CUtensorMap>* group_maps = nullptr,
                       const std::vector<CUtensorMap>* sketch_maps = nullptr) {
    const size_t bytes = pl.upload_bytes;
    char* host = nullptr;
    fm_status st = staging(c, bytes, &host);
    if (st != FM_OK) return st;
    memcpy(host + pl.desc_off, ds.data(), sizeof(FrameDesc) * ds.size());
    if (!maps.empty()) memcpy(host + pl.tmap_off, maps.data(), sizeof(CUtensorMap) * maps.size());
    if (group_maps && !group_maps->empty())
        memcpy(host + pl.tmap_off + sizeof(CUtensorMap) * ds.size(), group_maps->data(),
               sizeof(CUtensorMap) * group_maps->size());
    if (sketch_maps && !sketch_maps->empty())  // [2n, 6n): sketch R, B rows, raw R, split B rows
        memcpy(host + pl.tmap_off + sizeof(CUtensorMap) * 2 * ds.size(), sketch_maps->data(),
               sizeof(CUtensorMap) * sketch_maps->size());
    std::vector<GridDesc> g = pl.grids;
    for (size_t i = 0; i < g.size(); ++i) g[i].qtab = reinterpret_cast<float2*>(c->arena + pl.qtab[i]);
    if (!g.empty()) memcpy(host + pl.grid_off, g.data(), sizeof(GridDesc) * g.size());
    if (!pl.cov.items.empty())
        memcpy(host + pl.cov_items_off, pl.cov.items.data(), sizeof(fm::CovItem) * pl.cov.items.size());
    for (size_t k = 0; k < pl.pos_tab.size(); ++k) {
        const size_t end = k + 1 < pl.pos_host_at.size() ? pl.pos_host_at[k + 1] : pl.pos_host.size();
        memcpy(host + pl.pos_tab[k], pl.pos_host.data() + pl.pos_host_at[k], sizeof(float2) * (end - pl.pos_host_at[k]));
    }
    st = upload(c, host, c->arena, bytes, s);
    if (st != FM_OK) return st;
    *dd = reinterpret_cast<FrameDesc*>(c->arena + pl.desc_off);
    *dg = reinterpret_cast<GridDesc*>(c->arena + pl.grid_off);
    return FM_OK;
}

// Which kernels a sketch pass needs (bits of RunPrep::tc_pass).
enum : char { kPassPlain = 1, kPassSplit = 2, kPassDense = 4 };

// The fast-MUSIC chain from R (already formed) to U_s.
// tc_pass[p]: the kPass* bits of sketch pass p; sk_maps: n maps over R, n over the
// B rows, n over R in raw boxes, n over the split B rows.  Without them every
// product runs on the CUDA cores.
fm_status run_subspace_chain(fm_ctx* c, FrameDesc* dd, int n, const Maxes& mx, cudaStream_t s,
                             const char* sk_maps = nullptr, const std::vector<char>* tc_pass = nullptr,
                             bool prep_late = true) {
    auto sketch = [&](int p) {
        const bool tc = sk_maps && tc_pass;
        const char bits = tc ? (*tc_pass)[p] : (char)((p > 0 || mx.any_projection) ? kPassDense : 0);
        // Omega: only frames whose first product runs on the CUDA cores need omega_kernel (the
        // B-row preparation of the tensor-core sketch generates the others' Omega)
        cudaError_t e = fm::launch_sketch(dd, n, mx.M, mx.l, p, p == 0 && mx.any_sampling,
                                          p == 0 && mx.any_projection && (bits & kPassDense) != 0,
                                          (bits & kPassDense) != 0, s);
        if (e == cudaSuccess && (bits & (kPassPlain | kPassSplit))) {
            const size_t m = sizeof(CUtensorMap) * (size_t)n;
            e = fm::launch_sketch_tc(dd, n, mx.M, mx.l, p, (bits & kPassPlain) != 0, (bits & kPassSplit) != 0, sk_maps,
                                     sk_maps + m, sk_maps + 2 * m, sk_maps + 3 * m, s, p == 0 || prep_late);
        }
        return e;
    };
    fm_status st = stage(c, kStSketch, s, [&] { return sketch(0); });
    if (st != FM_OK) return st;
    for (int p = 1; p <= mx.t; ++p) {
        st = stage(c, kStOrth, s, [&] { return fm::launch_orth(dd, n, mx.M, mx.l, p, s); });
        if (st != FM_OK) return st;
        st = stage(c, kStSketch, s, [&] { return sketch(p); });
        if (st != FM_OK) return st;
    }
    if (mx.any_refine) {  // V = orth(C), then C = X (X^H V) / T in FP32 (frames with refine only)
        st = stage(c, kStOrth, s, [&] { return fm::launch_orth(dd, n, mx.M, mx.l, -1, s); });
        if (st != FM_OK) return st;
        st = stage(c, kStRefine, s, [&] { return fm::launch_refine(dd, n, mx.M, mx.T, s); });
        if (st != FM_OK) return st;
    }
    return stage(c, kStFinal, s, [&] { return fm::launch_final(dd, n, mx.M, mx.l, s); });
}

}  // namespace

// =================================================================== ABI ====
extern "C" {

fm_status fm_create(fm_ctx** ctx, size_t workspace_budget_bytes, int device) {
    if (!ctx) return FM_ERR_INVALID_ARG;
    *ctx = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return FM_ERR_CUDA;
    fm_ctx* c = new fm_ctx();
    c->device = device;
    c->budget = workspace_budget_bytes ? workspace_budget_bytes : ((size_t)16 << 30);
    if (cudaSetDevice(device) != cudaSuccess) {
        delete c;
        return FM_ERR_CUDA;
    }
    *ctx = c;
    return FM_OK;
}

fm_status fm_destroy(fm_ctx* c) {
    if (!c) return FM_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    for (fm_ctx::Slot* sl : c->slots) {
        if (sl->stream) cudaStreamSynchronize(sl->stream);
        if (sl->sub) fm_destroy(sl->sub);  // frees its workspace on sl->stream
        if (sl->stream) cudaStreamSynchronize(sl->stream);
        if (sl->ev) cudaEventDestroy(sl->ev);
        if (sl->stream) cudaStreamDestroy(sl->stream);
        delete sl;
    }
    for (fm_ctx::HostSlot& h : c->hslot) {
        if (h.d2h) cudaEventSynchronize(h.d2h);
        if (h.buf) cudaFree(h.buf);
        if (h.tab) cudaFreeHost(h.tab);
        if (h.h2d) cudaEventDestroy(h.h2d);
        if (h.comp) cudaEventDestroy(h.comp);
        if (h.d2h) cudaEventDestroy(h.d2h);
    }
    for (cudaStream_t hs : {c->s_h2d, c->s_comp, c->s_d2h})
        if (hs) {
            cudaStreamSynchronize(hs);
            cudaStreamDestroy(hs);
        }
    for (cudaEvent_t e : c->staging_done)
        if (e) {
            cudaEventSynchronize(e);
            cudaEventDestroy(e);
        }
    for (TimedEvent& t : c->pending) {
        cudaEventSynchronize(t.b);
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    for (cudaEvent_t e : c->pool) cudaEventDestroy(e);
    if (c->arena) {
        cudaDeviceSynchronize();
        if (c->arena_stream)
            cudaFreeAsync(c->arena, c->arena_stream);
        else
            cudaFree(c->arena);
    }
    for (char* h : c->pinned)
        if (h) cudaFreeHost(h);
    delete c;
    return FM_OK;
}

const char* fm_last_error(const fm_ctx* c) { return c ? c->err.c_str() : "null context"; }

// The order fm_run processes frames in: the frames of each tensor-core scan group (same
// M, ncols, prec, grid and geometry) next to each other, otherwise the caller's order.
static std::vector<int> run_order(const fm_frame* frames, int n) {
    std::vector<int> order(n);
    for (int b = 0; b < n; ++b) order[b] = b;
    const std::vector<int> geo = geometry_ids(frames, n);
    auto key = [&](int b) {
        const fm_frame& f = frames[b];
        return std::make_tuple(f.arr.M, ncols_of(f.p), f.p.prec, f.grid.theta0_deg, f.grid.step_deg, grid_spacing(f),
                               f.grid.L, geo[b]);
    };
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return key(x) < key(y); });
    return order;
}

// Workspace of fm_run for these (valid) frames; without the covariance's split tiles
// when split is false (then a batch of such frames needs at most the sum of their own
// figures plus cov_split_cap_bytes).
static size_t workspace_bytes(const fm_frame* frames, int n, bool split) {
    const std::vector<int> order = run_order(frames, n);
    std::vector<fm_frame> sorted(n);
    for (int k = 0; k < n; ++k) sorted[k] = frames[order[k]];
    return plan_frames(sorted.data(), n, true, true, true, true, split).total;
}

size_t fm_workspace_bytes(const fm_frame* frames, int n) {
    if (!frames || n < 1) return 0;
    for (int b = 0; b < n; ++b)
        if (check_frame(frames[b])) return 0;
    return workspace_bytes(frames, n, true);
}

// ---- fm_run, split into host preparation and the device chain -----------------
// Frames are processed in an order that puts the frames of each tensor-core
// scan group (same M, ncols, grid, prec) next to each other; order[k] is the
// caller's index of the k-th frame.
struct RunPrep {
    int n = 0;
    Plan pl;
    std::vector<int> order;
    Maxes mx;
    bool cov_tc = false, scan_tc = false, scan_simt = true, any_repack = false;
    std::vector<char> group_tc;  // per scan group: runs on the tensor cores
    std::vector<char> tc_pass;   // per sketch pass: kPass* bits of the kernels it needs
    bool prep_late = true;       // a tensor-core frame needs the B-row kernel at passes >= 1
    FrameDesc* dd = nullptr;
    GridDesc* dg = nullptr;
};

static fm_status prepare_run(fm_ctx* c, const fm_frame* frames, int n, cudaStream_t s, RunPrep& rp) {
    rp.n = n;
    rp.order = run_order(frames, n);
    std::vector<fm_frame> sorted(n);
    for (int k = 0; k < n; ++k) sorted[k] = frames[rp.order[k]];
    // a serving slot shares the GPU with the other slots' batches, so its covariance
    // does not split tiles to fill the SMs by itself
    rp.pl = plan_frames(sorted.data(), n, true, true, true, true, c->arena_stream == nullptr);
    const Plan& pl = rp.pl;
    fm_status st = ensure_arena(c, pl.total);
    if (st != FM_OK) return st;
    std::vector<FrameDesc> ds(n);
    c->last_us.assign(n, std::make_tuple(SIZE_MAX, 0, 0));
    for (int k = 0; k < n; ++k) {
        FrameDesc d = make_desc(sorted[k]);
        d.R = reinterpret_cast<float2*>(c->arena + pl.R[k]);
        d.C = reinterpret_cast<float2*>(c->arena + pl.C[k]);
        d.V = reinterpret_cast<float2*>(c->arena + pl.V[k]);
        d.idx = reinterpret_cast<int*>(c->arena + pl.idx[k]);
        d.Us = reinterpret_cast<float2*>(c->arena + pl.Us[k]);
        d.Y = pl.Y[k] != SIZE_MAX ? reinterpret_cast<float2*>(c->arena + pl.Y[k]) : nullptr;
        if (pl.Bsk[k] != SIZE_MAX && c->sketch_path != FM_COV_SIMT) {
            d.Bsk = reinterpret_cast<float*>(c->arena + pl.Bsk[k]);
            d.sketch_tc = 1;
        }
        if (pl.Xpad[k] != SIZE_MAX && c->cov_path != FM_COV_SIMT) {
            d.Xin = d.X;
            d.ldx_in = d.ldx;
            d.X = reinterpret_cast<const float2*>(c->arena + pl.Xpad[k]);
            d.ldx = d.T + (d.T & 1);
            rp.any_repack = true;
        }
        d.sweep_cap = c->sweep_cap;
        if (pl.fix[k] != SIZE_MAX) {
            d.fix_count = reinterpret_cast<int*>(c->arena + pl.fix[k]);
            d.fix_list = d.fix_count + 1;
        }
        c->last_us[rp.order[k]] = std::make_tuple(pl.Us[k], d.M, d.ncols);
        d.qtab = reinterpret_cast<float2*>(c->arena + pl.qtab[pl.grid_of[k]]);
        if (pl.geom_of[k]) d.pos = reinterpret_cast<const float2*>(c->arena + pl.pos_tab[pl.geom_of[k] - 1]);
        ds[k] = d;
    }
    std::vector<CUtensorMap> maps;
    st = choose_cov_path(c, ds, maps, &rp.cov_tc);
    if (st != FM_OK) return st;
    // tensor-core sketch: maps over R and the B rows of every frame that takes it
    std::vector<CUtensorMap> skmaps(4 * (size_t)n);
    memset(skmaps.data(), 0, sizeof(CUtensorMap) * skmaps.size());
    rp.tc_pass.assign(9, 0);
    int n_sk_tc = 0, n_sk_any = 0;
    // the power-step orthonormalisation writes the B rows of passes >= 1 where its clusters
    // split the frame's rows into whole chunks of the split layout
    const Maxes mx0 = maxes_of(ds);
    const int onc = mx0.t >= 1 ? fm::orth_cluster_size(mx0.M, mx0.l, n) : 0;
    rp.prep_late = false;
    for (int k = 0; k < n; ++k) {
        FrameDesc& d = ds[k];
        if (d.sketch_tc && !encode_sketch_tmaps(d, &skmaps[k], &skmaps[n + k], &skmaps[2 * n + k], &skmaps[3 * n + k]))
            d.sketch_tc = 0;  // the CUDA-core sketch takes every pass of this frame
        d.bsk_orth_nc = (d.sketch_tc && d.t >= 1 && onc > 0 && fm::brows_by_cluster(d.M, onc)) ? onc : 0;
        if (d.sketch_tc && d.t >= 1 && d.bsk_orth_nc == 0) rp.prep_late = true;
        bool has_product = false;
        for (int p = 0; p <= d.t; ++p) {
            if (!fm::sketch_on_tc(d.method, p)) continue;  // sampling, pass 0: a gather
            has_product = true;
            if (!d.sketch_tc)
                rp.tc_pass[p] |= kPassDense;
            else
                rp.tc_pass[p] |= fm::sketch_split(d.prec, d.t, p) ? kPassSplit : kPassPlain;
        }
        n_sk_any += has_product;
        n_sk_tc += has_product && d.sketch_tc;
    }
    if (c->sketch_path == FM_COV_TC && n_sk_tc < n_sk_any)
        return fail(c, FM_ERR_INVALID_ARG, "tensor-core sketch needs an even M (16-byte aligned rows of R)");
    c->last_sketch_path = n_sk_tc == n_sk_any ? FM_COV_TC : (n_sk_tc == 0 ? FM_COV_SIMT : FM_COV_AUTO);
    // scan: one batched tensor-core launch per scan group that fills at least a
    // quarter of the kernel's 512-row B tile (FM_COV_TC: every group), the CUDA-core
    // scan for the other frames, then the CUDA-core main-lobe recompute of the
    // tensor-core frames
    std::vector<CUtensorMap> gmaps(pl.scan_groups.size());
    rp.group_tc.assign(pl.scan_groups.size(), 0);
    int n_tc = 0;
    for (size_t g = 0; g < pl.scan_groups.size(); ++g) {
        const Plan::ScanGroup& sg = pl.scan_groups[g];
        const int fpc = 256 / fm::scan_tc_ncp(sg.nc);  // frames per CTA
        bool use = c->scan_path == FM_COV_TC || (c->scan_path == FM_COV_AUTO && 4 * sg.nf >= fpc);
        if (use) {
            use = encode_bprep_tmap(reinterpret_cast<float*>(c->arena + sg.bprep_off), sg.rows, sg.rowlen, &gmaps[g]);
            if (!use && c->scan_path == FM_COV_TC)
                return fail(c, FM_ERR_INVALID_ARG, "tensor-core scan: tensor map encoding failed");
        }
        rp.group_tc[g] = use;
        if (use) {
            n_tc += sg.nf;
            for (int k = sg.f0; k < sg.f0 + sg.nf; ++k) ds[k].scan_tc = 1;
        }
    }
    rp.scan_tc = n_tc > 0;
    rp.scan_simt = n_tc < n;
    c->last_scan_path = n_tc == n ? FM_COV_TC : (n_tc == 0 ? FM_COV_SIMT : FM_COV_AUTO);
    st = upload_descs(c, pl, ds, maps, s, &rp.dd, &rp.dg, rp.scan_tc ? &gmaps : nullptr, &skmaps);
    if (st != FM_OK) return st;
    rp.mx = maxes_of(ds);
    return FM_OK;
}

static fm_status enqueue_run(fm_ctx* c, const RunPrep& rp, cudaStream_t s) {
    const Plan& pl = rp.pl;
    const Maxes& mx = rp.mx;
    FrameDesc* dd = rp.dd;
    const int n = rp.n, ng = (int)pl.grids.size();
    int* counters = pl.cov.n_split ? reinterpret_cast<int*>(c->arena + pl.cov_cnt_off) : nullptr;
    fm_status st = stage(c, kStGrid, s, [&] {
        return fm::launch_grid_table(rp.dg, ng, mx.L, dd, n, counters, pl.cov.n_split, s);
    });
    if (st != FM_OK) return st;
    if (rp.any_repack) {  // frames whose X TMA cannot read get a padded copy first
        st = stage(c, kStCov, s, [&] { return fm::launch_repack(dd, n, mx.M, mx.T, s); });
        if (st != FM_OK) return st;
    }
    st = launch_cov(c, rp.cov_tc, dd, c->arena + pl.tmap_off,
                    reinterpret_cast<const fm::CovItem*>(c->arena + pl.cov_items_off), (int)pl.cov.items.size(),
                    pl.cov.n_split ? reinterpret_cast<float2*>(c->arena + pl.cov_part_off) : nullptr, counters, n, mx.M,
                    s);
    if (st != FM_OK) return st;
    st = run_subspace_chain(c, dd, n, mx, s, c->arena + pl.tmap_off + sizeof(CUtensorMap) * 2 * (size_t)n,
                            &rp.tc_pass, rp.prep_late);
    if (st != FM_OK) return st;
    st = stage(c, kStScan, s, [&] {
        if (rp.scan_simt) {  // frames without a tensor-core group (the kernel skips the others)
            cudaError_t e = fm::launch_scan(dd, n, mx.L, mx.M, mx.kpad, mx.scan_smem, s);
            if (e != cudaSuccess) return e;
        }
        if (rp.scan_tc) {
            for (size_t g = 0; g < pl.scan_groups.size(); ++g) {
                if (!rp.group_tc[g]) continue;
                const Plan::ScanGroup& sg = pl.scan_groups[g];
                float* bp = reinterpret_cast<float*>(c->arena + sg.bprep_off);
                const char* bmap_dev = c->arena + pl.tmap_off + sizeof(CUtensorMap) * ((size_t)n + g);
                cudaError_t e = fm::launch_scan_tc(dd + sg.f0, sg.nf, sg.M, sg.nc, sg.L, sg.prec,
                                                   pl.geom_of[sg.f0] != 0, bp, bmap_dev, s);
                if (e != cudaSuccess) return e;
            }
            // main-lobe angles again on the FP32 CUDA cores (see scan_kernel<..., FIXUP>)
            return fm::launch_scan_fixup(dd, n, mx.L, mx.M, mx.kpad, mx.scan_smem, s);
        }
        return cudaSuccess;
    });
    if (st != FM_OK) return st;
    return stage(c, kStPeaks, s, [&] { return fm::launch_peaks(dd, n, mx.K, mx.L, s); });
}

fm_status fm_run(fm_ctx* c, const fm_frame* frames, int n, fm_stream stream) {
    if (!c) return FM_ERR_INVALID_ARG;
    if (!frames || n < 1) return fail(c, FM_ERR_INVALID_ARG, "no frames");
    for (int b = 0; b < n; ++b) {
        const char* why = check_frame(frames[b]);
        if (why) return fail(c, FM_ERR_INVALID_ARG, "frame %d: %s", b, why);
    }
    fm_status st = set_device(c);
    if (st != FM_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    RunPrep rp;
    st = prepare_run(c, frames, n, s, rp);
    if (st != FM_OK) return st;
    return enqueue_run(c, rp, s);
}

// ---- fm_run with host buffers ---------------------------------------------------
// Three context streams: host -> device copies, the chain, device -> host copies,
// chained by events, with two device staging slots so that the copies of one
// call overlap the chain of the previous one.
fm_status fm_run_host(fm_ctx* c, const fm_frame* frames, int n, fm_stream stream) {
    if (!c) return FM_ERR_INVALID_ARG;
    if (!frames || n < 1) return fail(c, FM_ERR_INVALID_ARG, "fm_run_host: no frames");
    for (int b = 0; b < n; ++b) {
        const char* why = check_frame(frames[b]);
        if (why) return fail(c, FM_ERR_INVALID_ARG, "fm_run_host: frame %d: %s", b, why);
    }
    fm_status st = set_device(c);
    if (st != FM_OK) return st;
    cudaError_t e = cudaSuccess;
    for (cudaStream_t* hs : {&c->s_h2d, &c->s_comp, &c->s_d2h})
        if (!*hs && (e = cudaStreamCreateWithFlags(hs, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(c, e, "cudaStreamCreate");
    fm_ctx::HostSlot& h = c->hslot[c->hnext];
    c->hnext ^= 1;
    for (cudaEvent_t* ev : {&h.h2d, &h.comp, &h.d2h})
        if (!*ev && (e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(c, e, "cudaEventCreate");
    // device staging layout: every frame's packed X (M x T, rows padded to an even
    // length) back to back, so that frames adjacent in host memory arrive in one copy;
    // then every output; then the table of output copies
    std::vector<size_t> xo(n), po(n), dbo(n), io(n), dgo(n), no(n), so(n);
    size_t off = 0;
    for (int b = 0; b < n; ++b) {
        const fm_frame& f = frames[b];
        xo[b] = off;
        off += 8 * (size_t)f.arr.M * (size_t)(f.T + (f.T & 1));  // a multiple of 16 bytes
    }
    off = aup(off);
    int n_out = 0;
    for (int b = 0; b < n; ++b) {
        const fm_frame& f = frames[b];
        const size_t K = (size_t)f.p.K, L = (size_t)f.grid.L;
        po[b] = off;
        off = aup(off + 4 * L);
        dbo[b] = off;
        if (f.P_db_out) off = aup(off + 4 * L);
        io[b] = off;
        off = aup(off + 4 * K);
        dgo[b] = off;
        off = aup(off + 4 * K);
        no[b] = off;
        off = aup(off + 4);
        so[b] = off;
        off = aup(off + 4);
        n_out += 4 + (f.P_db_out ? 1 : 0) + (f.status ? 1 : 0);
    }
    const size_t tab_off = off;
    off = aup(off + sizeof(fm::CopyEntry) * (size_t)n_out);
    if (off > h.bytes) {
        if (h.used) cudaEventSynchronize(h.d2h);  // the slot's previous call is done with it
        if (h.buf) cudaFree(h.buf);
        h.buf = nullptr;
        h.bytes = 0;
        e = cudaMalloc(&h.buf, off + off / 4);
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaMalloc(host-run staging)");
        h.bytes = off + off / 4;
    }
    cudaStream_t us = reinterpret_cast<cudaStream_t>(stream);
    // copies in: once this slot's previous results have left (the host X must hold its
    // data when the call is made; waiting on `stream` here would also wait for the
    // previous call's copies out, which `stream` is made to wait for, and serialise)
    if (h.used) cudaStreamWaitEvent(c->s_h2d, h.d2h, 0);
    std::vector<fm_frame> dev(frames, frames + n);
    // one copy per run of frames that are contiguous both in host memory and here
    const char* run_src = nullptr;
    size_t run_dst = 0, run_bytes = 0;
    auto flush = [&]() -> cudaError_t {
        if (!run_bytes) return cudaSuccess;
        const cudaError_t r = cudaMemcpyAsync(h.buf + run_dst, run_src, run_bytes, cudaMemcpyHostToDevice, c->s_h2d);
        run_bytes = 0;
        return r;
    };
    for (int b = 0; b < n; ++b) {
        const fm_frame& f = frames[b];
        const size_t row = 8 * (size_t)f.T;
        const int64_t ldd = f.T + (f.T & 1);
        if (f.ldx == f.T && ldd == f.T) {  // one contiguous block
            const char* src = reinterpret_cast<const char*>(f.X);
            const size_t bytes = row * (size_t)f.arr.M;
            if (run_bytes && src == run_src + run_bytes && xo[b] == run_dst + run_bytes) {
                run_bytes += bytes;
            } else {
                e = flush();
                run_src = src;
                run_dst = xo[b];
                run_bytes = bytes;
            }
        } else {
            e = flush();
            if (e == cudaSuccess)
                e = cudaMemcpy2DAsync(h.buf + xo[b], 8 * (size_t)ldd, f.X, 8 * (size_t)f.ldx, row, (size_t)f.arr.M,
                                      cudaMemcpyHostToDevice, c->s_h2d);
        }
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemcpyAsync(X)");
        dev[b].X = h.buf + xo[b];
        dev[b].ldx = ldd;
        dev[b].P_out = reinterpret_cast<float*>(h.buf + po[b]);
        dev[b].P_db_out = f.P_db_out ? reinterpret_cast<float*>(h.buf + dbo[b]) : nullptr;
        dev[b].peak_idx = reinterpret_cast<int*>(h.buf + io[b]);
        dev[b].peak_deg = reinterpret_cast<float*>(h.buf + dgo[b]);
        dev[b].n_peaks = reinterpret_cast<int*>(h.buf + no[b]);
        dev[b].status = reinterpret_cast<int*>(h.buf + so[b]);
    }
    e = flush();
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemcpyAsync(X)");
    cudaEventRecord(h.h2d, c->s_h2d);
    // the chain
    cudaStreamWaitEvent(c->s_comp, h.h2d, 0);
    RunPrep rp;
    st = prepare_run(c, dev.data(), n, c->s_comp, rp);
    if (st != FM_OK) return st;
    st = enqueue_run(c, rp, c->s_comp);
    if (st != FM_OK) return st;
    cudaEventRecord(h.comp, c->s_comp);
    // copies out: where the device writes host memory through its host address, one
    // kernel scatters every output (after one upload of the copy table); else one
    // copy per output buffer
    cudaStreamWaitEvent(c->s_d2h, h.comp, 0);
    if (c->host_direct < 0) {
        int pageable = 0;
        cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, c->device);
        c->host_direct = pageable ? 1 : 0;
    }
    std::vector<fm::CopyEntry> tab;
    tab.reserve((size_t)n_out);
    for (int b = 0; b < n; ++b) {
        const fm_frame& f = frames[b];
        const int64_t L = f.grid.L, K = f.p.K;
        tab.push_back({h.buf + po[b], f.P_out, 4 * L});
        if (f.P_db_out) tab.push_back({h.buf + dbo[b], f.P_db_out, 4 * L});
        tab.push_back({h.buf + io[b], f.peak_idx, 4 * K});
        tab.push_back({h.buf + dgo[b], f.peak_deg, 4 * K});
        tab.push_back({h.buf + no[b], f.n_peaks, 4});
        if (f.status) tab.push_back({h.buf + so[b], f.status, 4});
    }
    bool direct = c->host_direct == 1;
    for (const fm::CopyEntry& t : tab) direct = direct && (reinterpret_cast<uintptr_t>(t.dst) % 4) == 0;
    if (direct) {
        if (h.used) cudaEventSynchronize(h.d2h);  // the slot's previous table upload is done
        if (h.tab_cap < tab.size()) {
            if (h.tab) cudaFreeHost(h.tab);
            h.tab = nullptr;
            h.tab_cap = 0;
            e = cudaMallocHost(reinterpret_cast<void**>(&h.tab), sizeof(fm::CopyEntry) * tab.size());
            if (e != cudaSuccess) return cuda_fail(c, e, "cudaMallocHost(copy table)");
            h.tab_cap = tab.size();
        }
        memcpy(h.tab, tab.data(), sizeof(fm::CopyEntry) * tab.size());
        fm::CopyEntry* dtab = reinterpret_cast<fm::CopyEntry*>(h.buf + tab_off);
        e = cudaMemcpyAsync(dtab, h.tab, sizeof(fm::CopyEntry) * tab.size(), cudaMemcpyHostToDevice, c->s_d2h);
        if (e == cudaSuccess) e = fm::launch_scatter(dtab, (int)tab.size(), c->s_d2h);
        if (e != cudaSuccess) return cuda_fail(c, e, "output scatter");
        c->launches += 1;
    } else {
        for (const fm::CopyEntry& t : tab) {
            e = cudaMemcpyAsync(t.dst, t.src, (size_t)t.bytes, cudaMemcpyDeviceToHost, c->s_d2h);
            if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemcpyAsync(outputs)");
        }
    }
    cudaEventRecord(h.d2h, c->s_d2h);
    h.used = true;
    e = cudaStreamWaitEvent(us, h.d2h, 0);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamWaitEvent");
    return FM_OK;
}

// ---- autotuning of the kernel paths -------------------------------------------
// Times fm_run on the caller's frames for every combination of covariance path
// and scan path that these frames can take (tensor-core 128 x 256 tiles or
// CUDA-core tiles), keeps the fastest in the context and reports it.
fm_status fm_autotune(fm_ctx* c, const fm_frame* frames, int n, fm_stream stream, int reps, int* cov_path,
                      int* scan_path, float* best_ms) {
    if (!c) return FM_ERR_INVALID_ARG;
    if (!frames || n < 1 || reps < 1) return fail(c, FM_ERR_INVALID_ARG, "fm_autotune: no frames or reps < 1");
    fm_status st = set_device(c);
    if (st != FM_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int saved_cov = c->cov_path, saved_scan = c->scan_path;
    const unsigned saved_timing = c->timing;
    c->timing = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = -1.f;
    int bc = saved_cov, bs = saved_scan;
    const int paths[2] = {FM_COV_TC, FM_COV_SIMT};
    for (int cp : paths)
        for (int sp : paths) {
            c->cov_path = cp;
            c->scan_path = sp;
            if (fm_run(c, frames, n, stream) != FM_OK) continue;  // this path is not open to these frames
            cudaEventRecord(e0, s);
            bool ok = true;
            for (int r = 0; r < reps && ok; ++r) ok = fm_run(c, frames, n, stream) == FM_OK;
            cudaEventRecord(e1, s);
            if (!ok || cudaEventSynchronize(e1) != cudaSuccess) continue;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= (float)reps;
            if (best < 0.f || ms < best) {
                best = ms;
                bc = cp;
                bs = sp;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->timing = saved_timing;
    c->cov_path = bc;
    c->scan_path = bs;
    if (best < 0.f) {
        c->cov_path = saved_cov;
        c->scan_path = saved_scan;
        return fail(c, FM_ERR_INVALID_ARG, "fm_autotune: no path ran these frames");
    }
    c->err.clear();
    if (cov_path) *cov_path = bc;
    if (scan_path) *scan_path = bs;
    if (best_ms) *best_ms = best;
    return FM_OK;
}

// ---- CUDA graphs ------------------------------------------------------------
// A graph owns a private context (its own workspace and descriptors, prepared
// once) and the instantiated capture of the chain's kernel launches.
struct fm_graph {
    fm_ctx* parent = nullptr;
    fm_ctx* sub = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t kernels = 0;  // kernel launches per graph launch
};

fm_status fm_graph_create(fm_ctx* c, const fm_frame* frames, int n, fm_graph** out) {
    if (!c) return FM_ERR_INVALID_ARG;
    if (!out || !frames || n < 1) return fail(c, FM_ERR_INVALID_ARG, "fm_graph_create: no frames");
    *out = nullptr;
    for (int b = 0; b < n; ++b) {
        const char* why = check_frame(frames[b]);
        if (why) return fail(c, FM_ERR_INVALID_ARG, "fm_graph_create: frame %d: %s", b, why);
    }
    fm_status st = set_device(c);
    if (st != FM_OK) return st;
    fm_graph* g = new fm_graph();
    g->parent = c;
    cudaStream_t cs = nullptr;
    auto bail = [&](fm_status code) {
        if (cs) cudaStreamDestroy(cs);
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
        if (g->sub) {
            if (!g->sub->err.empty()) c->err = g->sub->err;  // the failure was recorded on the graph's context
            fm_destroy(g->sub);
        }
        delete g;
        return code;
    };
    if (fm_create(&g->sub, c->budget, c->device) != FM_OK) return bail(fail(c, FM_ERR_CUDA, "fm_graph_create: context"));
    g->sub->cov_path = c->cov_path;
    g->sub->scan_path = c->scan_path;
    g->sub->sketch_path = c->sketch_path;
    g->sub->sweep_cap = c->sweep_cap;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaStreamCreate"));
    RunPrep rp;
    st = prepare_run(g->sub, frames, n, cs, rp);
    if (st != FM_OK) return bail(st);
    st = enqueue_run(g->sub, rp, cs);  // one plain run: uploads land, kernel attributes are set
    if (st != FM_OK) return bail(st);
    e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaStreamSynchronize"));
    const uint64_t l0 = g->sub->launches;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaStreamBeginCapture"));
    st = enqueue_run(g->sub, rp, cs);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(cs, &graph);
    g->graph = graph;
    if (st != FM_OK) return bail(st);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaStreamEndCapture"));
    g->kernels = g->sub->launches - l0;
    e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaGraphInstantiate"));
    cudaStreamDestroy(cs);
    *out = g;
    return FM_OK;
}

fm_status fm_graph_launch(fm_graph* g, fm_stream stream) {
    if (!g) return FM_ERR_INVALID_ARG;
    fm_status st = set_device(g->parent);
    if (st != FM_OK) return st;
    cudaError_t e = cudaGraphLaunch(g->exec, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(g->parent, e, "cudaGraphLaunch");
    g->parent->launches += g->kernels;
    return FM_OK;
}

fm_status fm_graph_destroy(fm_graph* g) {
    if (!g) return FM_ERR_INVALID_ARG;
    cudaSetDevice(g->parent->device);
    cudaDeviceSynchronize();  // a launch may still be in flight
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    if (g->sub) fm_destroy(g->sub);
    delete g;
    return FM_OK;
}

fm_status fm_selftest_wait_timeout(fm_ctx* c, int* status, double limit_ms, fm_stream stream) {
    if (!c) return FM_ERR_INVALID_ARG;
    if (!status || !(limit_ms > 0.0) || limit_ms > 10000.0)
        return fail(c, FM_ERR_INVALID_ARG, "fm_selftest_wait_timeout: status NULL or limit_ms not in (0, 1e4]");
    fm_status st = set_device(c);
    if (st != FM_OK) return st;
    int khz = 0;
    cudaError_t e = cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaDeviceGetAttribute(clock rate)");
    const long long cycles = (long long)(limit_ms * (double)khz);
    st = stage(c, kStGrid, reinterpret_cast<cudaStream_t>(stream),
               [&] { return fm::launch_wait_timeout(status, cycles, reinterpret_cast<cudaStream_t>(stream)); });
    return st;
}

fm_status fm_run_subspace(fm_ctx* c, int frame, void* U, fm_stream stream) {
    if (!c) return FM_ERR_INVALID_ARG;
    if (!U || frame < 0 || frame >= (int)c->last_us.size() || std::get<0>(c->last_us[frame]) == SIZE_MAX)
        return fail(c, FM_ERR_INVALID_ARG, "fm_run_subspace: no frame %d in the last fm_run", frame);
    fm_status st = set_device(c);
    if (st != FM_OK) return st;
    const size_t bytes = sizeof(float2) * (size_t)std::get<1>(c->last_us[frame]) * std::get<2>(c->last_us[frame]);
    cudaError_t e = cudaMemcpyAsync(U, c->arena + std::get<0>(c->last_us[frame]), bytes, cudaMemcpyDeviceToDevice,
                                    reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemcpyAsync(U_s)");
    return FM_OK;
}

fm_status fm_covariance(fm_ctx* c, const void* X, int n, int M, int T, int64_t ldx, int64_t xstride, void* R,
                        int prec, fm_stream stream) {
    if (!c) return FM_ERR_INVALID_ARG;
    if (!X || !R || n < 1 || M < 1 || M > 65536 || T < 1 || ldx < T || xstride < (int64_t)(M - 1) * ldx + T)
        return fail(c, FM_ERR_INVALID_ARG, "fm_covariance: invalid shape or pointer");
    if (prec != FM_PREC_FP32 && prec != FM_PREC_TF32 && prec != FM_PREC_BF16)
        return fail(c, FM_ERR_INVALID_ARG, "fm_covariance: prec must be 0, 1 or 2");
    fm_status st = set_device(c);
    if (st != FM_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // uniform frames: the tiles in frame order, none split
    std::vector<fm::CovItem> items;
    {
        const int nt = (M + fm::kCovTile - 1) / fm::kCovTile, ns = (T + 15) / 16;
        for (int b = 0; b < n; ++b)
            for (int ti = 0; ti < nt; ++ti)
                for (int tj = ti; tj < nt; ++tj) items.push_back(fm::CovItem{b, ti, tj, 0, ns, -1, 0, 0, 1});
    }
    const size_t tmap_off = aup(sizeof(FrameDesc) * (size_t)n);
    const size_t items_off = aup(tmap_off + sizeof(CUtensorMap) * (size_t)n);
    const size_t bytes = items_off + sizeof(fm::CovItem) * items.size();
    st = ensure_arena(c, bytes);
    if (st != FM_OK) return st;
    std::vector<FrameDesc> ds(n);
    for (int b = 0; b < n; ++b) {
        FrameDesc d{};
        d.X = reinterpret_cast<const float2*>(X) + (int64_t)b * xstride;
        d.ldx = ldx;
        d.M = M;
        d.T = T;
        d.prec = prec;
        d.R = reinterpret_cast<float2*>(R) + (int64_t)b * M * M;
        ds[b] = d;
    }
    std::vector<CUtensorMap> maps;
    bool tc = false;
    st = choose_cov_path(c, ds, maps, &tc);
    if (st != FM_OK) return st;
    char* host = nullptr;
    st = staging(c, bytes, &host);
    if (st != FM_OK) return st;
    memcpy(host, ds.data(), sizeof(FrameDesc) * n);
    if (tc) memcpy(host + tmap_off, maps.data(), sizeof(CUtensorMap) * n);
    memcpy(host + items_off, items.data(), sizeof(fm::CovItem) * items.size());
    st = upload(c, host, c->arena, bytes, s);
    if (st != FM_OK) return st;
    FrameDesc* dd = reinterpret_cast<FrameDesc*>(c->arena);
    return launch_cov(c, tc, dd, c->arena + tmap_off, reinterpret_cast<const fm::CovItem*>(c->arena + items_off),
                      (int)items.size(), nullptr, nullptr, n, M, s);
}

fm_status fm_subspace(fm_ctx* c, const void* R, int n, int M, const fm_params* p, uint64_t frame_id0, void* U,
                      int* status, fm_stream stream) {
    if (!c) return FM_ERR_INVALID_ARG;
    if (!R || !U || !p || n < 1) return fail(c, FM_ERR_INVALID_ARG, "fm_subspace: NULL argument");
    if (p->refine) return fail(c, FM_ERR_INVALID_ARG, "fm_subspace: refine needs the snapshots X (use fm_run)");
    std::vector<fm_frame> fr(n);
    for (int b = 0; b < n; ++b) {
        fm_frame f{};
        f.X = R;  // placeholder for validation only
        f.T = 1;
        f.ldx = 1;
        f.arr.M = M;
        f.arr.d_wl = 0.5;
        f.grid.L = 1;
        f.grid.step_deg = 1.0;
        f.p = *p;
        f.frame_id = frame_id0 + (uint64_t)b;
        f.P_out = reinterpret_cast<float*>(U);
        f.peak_idx = status ? status : reinterpret_cast<int*>(U);
        f.peak_deg = f.P_out;
        f.n_peaks = f.peak_idx;
        const char* why = check_frame(f);
        if (why) return fail(c, FM_ERR_INVALID_ARG, "fm_subspace: %s", why);
        fr[b] = f;
    }
    fm_status st = set_device(c);
    if (st != FM_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Plan pl = plan_frames(fr.data(), n, false, true, false, false);
    st = ensure_arena(c, pl.total);
    if (st != FM_OK) return st;
    const int nc = ncols_of(*p);
    std::vector<FrameDesc> ds(n);
    for (int b = 0; b < n; ++b) {
        FrameDesc d = make_desc(fr[b]);
        d.X = nullptr;
        d.P = nullptr;
        d.peak_idx = nullptr;
        d.peak_deg = nullptr;
        d.n_peaks = nullptr;
        d.status = status ? status + b : nullptr;
        d.R = const_cast<float2*>(reinterpret_cast<const float2*>(R)) + (int64_t)b * M * M;
        d.C = reinterpret_cast<float2*>(c->arena + pl.C[b]);
        d.V = reinterpret_cast<float2*>(c->arena + pl.V[b]);
        d.idx = reinterpret_cast<int*>(c->arena + pl.idx[b]);
        d.Us = reinterpret_cast<float2*>(U) + (int64_t)b * M * nc;
        ds[b] = d;
    }
    if (status) {
        cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int) * (size_t)n, s);
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemsetAsync(status)");
    }
    FrameDesc* dd;
    GridDesc* dg;
    st = upload_descs(c, pl, ds, {}, s, &dd, &dg);
    if (st != FM_OK) return st;
    return run_subspace_chain(c, dd, n, maxes_of(ds), s);
}

static fm_status spectrum_impl(fm_ctx* c, const void* U, int n, const fm_array& arr, int ncols, const fm_grid* grid,
                               float* P, fm_stream stream, const char* name) {
    if (!c) return FM_ERR_INVALID_ARG;
    const int M = arr.M;
    if (!U || !grid || !P || n < 1 || M < 1 || M > fm::kMMax || ncols < 1 || ncols > fm::kKPadMax ||
        (size_t)M * (size_t)((ncols + 3) / 4 * 4) > 24576 || grid->L < 1 || grid->L > 65536 ||
        !std::isfinite(grid->theta0_deg) || !std::isfinite(grid->step_deg))
        return fail(c, FM_ERR_INVALID_ARG, "%s: invalid shape or pointer", name);
    if (arr.pos_wl) {
        for (int m = 0; m < M; ++m)
            if (!(std::fabs(arr.pos_wl[m]) <= 4096.0))
                return fail(c, FM_ERR_INVALID_ARG, "%s: positions must be finite with |x| <= 4096", name);
    } else if (!(arr.d_wl >= 0.0 && arr.d_wl <= 1.0)) {
        return fail(c, FM_ERR_INVALID_ARG, "%s: d_wl must be in (0, 1] (0 selects 0.5)", name);
    }
    fm_status st = set_device(c);
    if (st != FM_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    std::vector<fm_frame> fr(n);
    for (int b = 0; b < n; ++b) {
        fm_frame f{};
        f.arr = arr;
        f.grid = *grid;
        f.p.K = ncols;
        f.p.l = ncols;
        fr[b] = f;
    }
    Plan pl = plan_frames(fr.data(), n, false, false, false, true);
    st = ensure_arena(c, pl.total);
    if (st != FM_OK) return st;
    std::vector<FrameDesc> ds(n);
    for (int b = 0; b < n; ++b) {
        FrameDesc d = make_desc(fr[b]);
        d.ncols = d.kpad = ncols;
        d.Us = const_cast<float2*>(reinterpret_cast<const float2*>(U)) + (int64_t)b * M * ncols;
        d.P = P + (int64_t)b * grid->L;
        d.qtab = reinterpret_cast<float2*>(c->arena + pl.qtab[pl.grid_of[b]]);
        if (pl.geom_of[b]) d.pos = reinterpret_cast<const float2*>(c->arena + pl.pos_tab[pl.geom_of[b] - 1]);
        ds[b] = d;
    }
    FrameDesc* dd;
    GridDesc* dg;
    st = upload_descs(c, pl, ds, {}, s, &dd, &dg);
    if (st != FM_OK) return st;
    const Maxes mx = maxes_of(ds);
    st = stage(c, kStGrid, s,
               [&] { return fm::launch_grid_table(dg, (int)pl.grids.size(), mx.L, nullptr, 0, nullptr, 0, s); });
    if (st != FM_OK) return st;
    return stage(c, kStScan, s, [&] { return fm::launch_scan(dd, n, mx.L, mx.M, mx.kpad, mx.scan_smem, s); });
}

fm_status fm_spectrum(fm_ctx* c, const void* U, int n, int M, int ncols, double d_wl, const fm_grid* grid, float* P,
                      fm_stream stream) {
    fm_array arr{};
    arr.M = M;
    arr.d_wl = d_wl;
    return spectrum_impl(c, U, n, arr, ncols, grid, P, stream, "fm_spectrum");
}

fm_status fm_spectrum_array(fm_ctx* c, const void* U, int n, const fm_array* arr, int ncols, const fm_grid* grid,
                            float* P, fm_stream stream) {
    if (!c) return FM_ERR_INVALID_ARG;
    if (!arr) return fail(c, FM_ERR_INVALID_ARG, "fm_spectrum_array: arr is NULL");
    return spectrum_impl(c, U, n, *arr, ncols, grid, P, stream, "fm_spectrum_array");
}

fm_status fm_peaks(fm_ctx* c, const float* P, int n, int L, int K, const fm_grid* grid, int* peak_idx,
                   float* peak_deg, int* n_peaks, fm_stream stream) {
    if (!c) return FM_ERR_INVALID_ARG;
    if (!P || !grid || !peak_idx || !peak_deg || !n_peaks || n < 1 || L < 1 || L > 65536 || K < 1)
        return fail(c, FM_ERR_INVALID_ARG, "fm_peaks: invalid shape or pointer");
    fm_status st = set_device(c);
    if (st != FM_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t bytes = aup(sizeof(FrameDesc) * (size_t)n);
    st = ensure_arena(c, bytes);
    if (st != FM_OK) return st;
    std::vector<FrameDesc> ds(n);
    for (int b = 0; b < n; ++b) {
        FrameDesc d{};
        d.L = L;
        d.K = K;
        d.P = const_cast<float*>(P) + (int64_t)b * L;
        d.peak_idx = peak_idx + (int64_t)b * K;
        d.peak_deg = peak_deg + (int64_t)b * K;
        d.n_peaks = n_peaks + b;
        d.theta0 = grid->theta0_deg;
        d.step = grid->step_deg;
        ds[b] = d;
    }
    char* host = nullptr;
    st = staging(c, bytes, &host);
    if (st != FM_OK) return st;
    memcpy(host, ds.data(), sizeof(FrameDesc) * n);
    st = upload(c, host, c->arena, sizeof(FrameDesc) * n, s);
    if (st != FM_OK) return st;
    FrameDesc* dd = reinterpret_cast<FrameDesc*>(c->arena);
    return stage(c, kStPeaks, s, [&] { return fm::launch_peaks(dd, n, K, L, s); });
}

fm_status fm_test_matrix(fm_ctx* c, uint64_t seed, uint64_t frame_id, int M, int l, void* Pi, fm_stream stream) {
    if (!c) return FM_ERR_INVALID_ARG;
    if (!Pi || M < 1 || l < 1) return fail(c, FM_ERR_INVALID_ARG, "fm_test_matrix: invalid argument");
    fm_status st = set_device(c);
    if (st != FM_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = fm::launch_test_matrix(seed, frame_id, M, l, reinterpret_cast<float2*>(Pi), s);
    if (e != cudaSuccess) return cuda_fail(c, e, "test matrix launch");
    c->launches += 1;
    return FM_OK;
}

fm_status fm_sample_indices(fm_ctx* c, uint64_t seed, uint64_t frame_id, int M, int l, int* idx, fm_stream stream) {
    if (!c) return FM_ERR_INVALID_ARG;
    if (!idx || M < 1 || M > 65536 || l < 1 || l > M)
        return fail(c, FM_ERR_INVALID_ARG, "fm_sample_indices: invalid argument");
    fm_status st = set_device(c);
    if (st != FM_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = fm::launch_sample_indices(seed, frame_id, M, l, idx, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "sample indices launch");
    c->launches += 1;
    return FM_OK;
}

fm_status fm_set_timing(fm_ctx* c, int enable) {
    if (!c) return FM_ERR_INVALID_ARG;
    c->timing = enable != 0 ? (1u << FM_N_STAGES) - 1u : 0u;
    return FM_OK;
}

fm_status fm_set_timing_mask(fm_ctx* c, unsigned mask) {
    if (!c) return FM_ERR_INVALID_ARG;
    c->timing = mask & ((1u << FM_N_STAGES) - 1u);
    return FM_OK;
}

fm_status fm_stage_times(fm_ctx* c, double* total_ms, int* launches, int reset) {
    if (!c) return FM_ERR_INVALID_ARG;
    for (TimedEvent& t : c->pending) {
        cudaError_t e = cudaEventSynchronize(t.b);
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaEventSynchronize(stage)");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, t.a, t.b);
        c->stage_ms[t.stage] += ms;
        c->stage_n[t.stage] += 1;
        c->pool.push_back(t.a);
        c->pool.push_back(t.b);
    }
    c->pending.clear();
    for (int i = 0; i < FM_N_STAGES; ++i) {
        if (total_ms) total_ms[i] = c->stage_ms[i];
        if (launches) launches[i] = c->stage_n[i];
    }
    if (reset) {
        for (int i = 0; i < FM_N_STAGES; ++i) {
            c->stage_ms[i] = 0.0;
            c->stage_n[i] = 0;
        }
    }
    return FM_OK;
}

fm_status fm_set_cov_path(fm_ctx* c, int path) {
    if (!c) return FM_ERR_INVALID_ARG;
    if (path != FM_COV_AUTO && path != FM_COV_SIMT && path != FM_COV_TC)
        return fail(c, FM_ERR_INVALID_ARG, "unknown covariance path %d", path);
    c->cov_path = path;
    return FM_OK;
}

int fm_last_cov_path(const fm_ctx* c) { return c ? c->last_cov_path : 0; }

fm_status fm_set_scan_path(fm_ctx* c, int path) {
    if (!c) return FM_ERR_INVALID_ARG;
    if (path != FM_COV_AUTO && path != FM_COV_SIMT && path != FM_COV_TC)
        return fail(c, FM_ERR_INVALID_ARG, "unknown scan path %d", path);
    c->scan_path = path;
    return FM_OK;
}

int fm_last_scan_path(const fm_ctx* c) { return c ? c->last_scan_path : 0; }

fm_status fm_set_sketch_path(fm_ctx* c, int path) {
    if (!c) return FM_ERR_INVALID_ARG;
    if (path != FM_COV_AUTO && path != FM_COV_SIMT && path != FM_COV_TC)
        return fail(c, FM_ERR_INVALID_ARG, "unknown sketch path %d", path);
    c->sketch_path = path;
    return FM_OK;
}

int fm_last_sketch_path(const fm_ctx* c) { return c ? c->last_sketch_path : 0; }

fm_status fm_set_sweep_cap(fm_ctx* c, int cap) {
    if (!c) return FM_ERR_INVALID_ARG;
    if (cap < 0 || cap > 30) return fail(c, FM_ERR_INVALID_ARG, "sweep cap %d not in [0, 30]", cap);
    c->sweep_cap = cap;
    return FM_OK;
}

uint64_t fm_launch_count(const fm_ctx* c) { return c ? c->launches + c->serve_launches : 0; }

// ------------------------------------------------------------ serving ----
// Continuous batching.  A fixed set of slots (stream + private workspace) runs
// batches; whenever a slot is free, it takes the queued frames in arrival order,
// as many as fit (at most kServeMaxBatch, and the batch's workspace within what
// the budget leaves after the other slots' workspaces), and runs them as one
// fm_run batch.  Under light load a frame starts alone as soon as it arrives;
// under heavy load the queue grows while the slots are busy and the next batches
// are larger.  Frames that arrive while others run overlap with them on the GPU.
constexpr int kServeMaxSlots = 4;
constexpr int kServeMaxBatch = 64;

// Only for an idle slot (no work of its stream still reads the workspace).
static void release_arena(fm_ctx* sub) {
    cudaFreeAsync(sub->arena, sub->arena_stream);
    sub->arena = nullptr;
    sub->arena_bytes = 0;
}

static size_t serve_held(const fm_ctx* c) {
    size_t held = 0;
    for (const fm_ctx::Slot* sl : c->slots) held += sl->sub ? sl->sub->arena_bytes : 0;
    return held;
}

static void serve_progress(fm_ctx* c) {
    // retire finished slots
    // (any result but "not ready" ends the batch: an error fails its tickets, whose
    // fm_serve_poll then returns FM_ERR_CUDA, and is kept as the context's message)
    for (fm_ctx::Slot* sl : c->slots) {
        if (!sl->busy) continue;
        const cudaError_t q = cudaEventQuery(sl->ev);
        if (q == cudaErrorNotReady) continue;
        if (q != cudaSuccess) cuda_fail(c, q, "serving batch");
        for (uint64_t t : sl->tickets) c->done[t] = (q == cudaSuccess) ? 1 : -1;
        sl->tickets.clear();
        sl->busy = false;
    }
    std::vector<fm_frame> batch;
    while (!c->queue.empty()) {
        fm_ctx::Slot* pick = nullptr;  // the free slot with the largest workspace
        for (fm_ctx::Slot* sl : c->slots)
            if (!sl->busy && (!pick || sl->sub->arena_bytes > pick->sub->arena_bytes)) pick = sl;
        if (!pick && (int)c->slots.size() < kServeMaxSlots) {
            fm_ctx::Slot* sl = new fm_ctx::Slot();
            if (cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&sl->ev, cudaEventDisableTiming) != cudaSuccess ||
                fm_create(&sl->sub, c->budget, c->device) != FM_OK) {
                if (sl->ev) cudaEventDestroy(sl->ev);
                if (sl->stream) cudaStreamDestroy(sl->stream);
                delete sl;
                break;
            }
            sl->sub->arena_stream = sl->stream;
            sl->sub->cov_path = c->cov_path;
            sl->sub->scan_path = c->scan_path;
            sl->sub->sketch_path = c->sketch_path;
            sl->sub->sweep_cap = c->sweep_cap;
            c->slots.push_back(sl);
            pick = sl;
        }
        if (!pick) break;  // every slot busy: the queue waits and the next batch grows
        const size_t others = serve_held(c) - pick->sub->arena_bytes;
        const size_t room = c->budget > others ? c->budget - others : 0;
        batch.clear();
        // the sum of the frames' own workspaces plus the split-tile cap bounds a batch's
        // workspace; the exact plan is computed only once that cheap bound no longer fits
        const size_t avail = std::max(pick->sub->arena_bytes, room);
        const size_t cap = cov_split_cap_bytes(current_sm_count());
        size_t own = 0;  // the batch's frames' own workspaces, without split tiles
        for (const auto& q : c->queue) {
            if ((int)batch.size() == kServeMaxBatch) break;
            batch.push_back(q.frame);
            own += q.need;
            if (own + cap <= avail) continue;
            const size_t need = fm_workspace_bytes(batch.data(), (int)batch.size());
            if (need > avail) {  // the slot could not grow that far
                batch.pop_back();  // empty when not even the first frame fits
                break;
            }
        }
        pick->sub->arena_cap = room;
        if (batch.empty()) {
            // release the workspaces of the other idle slots, then retry; with none left
            // to release, wait for a busy slot to finish
            bool freed = false;
            for (fm_ctx::Slot* sl : c->slots)
                if (!sl->busy && sl != pick && sl->sub->arena) {
                    release_arena(sl->sub);
                    freed = true;
                }
            if (freed) continue;
            break;
        }
        fm_status st = fm_run(pick->sub, batch.data(), (int)batch.size(), reinterpret_cast<fm_stream>(pick->stream));
        pick->tickets.clear();
        for (size_t i = 0; i < batch.size(); ++i) {
            pick->tickets.push_back(c->queue.front().ticket);
            c->queue.pop_front();
        }
        if (st != FM_OK) {
            c->err = pick->sub->err;
            for (uint64_t t : pick->tickets) c->done[t] = -1;
            pick->tickets.clear();
            continue;
        }
        cudaEventRecord(pick->ev, pick->stream);
        pick->busy = true;
    }
    uint64_t n = 0;
    for (fm_ctx::Slot* sl : c->slots) n += sl->sub->launches;
    c->serve_launches = n;
}

fm_status fm_serve_submit(fm_ctx* c, const fm_frame* frame, uint64_t* ticket) {
    if (!c) return FM_ERR_INVALID_ARG;
    if (!frame || !ticket) return fail(c, FM_ERR_INVALID_ARG, "fm_serve_submit: NULL argument");
    const char* why = check_frame(*frame);
    if (why) return fail(c, FM_ERR_INVALID_ARG, "fm_serve_submit: %s", why);
    if (workspace_bytes(frame, 1, true) > c->budget)
        return fail(c, FM_ERR_OOM_BUDGET, "fm_serve_submit: frame needs more workspace than the budget");
    fm_status st = set_device(c);
    if (st != FM_OK) return st;
    *ticket = c->next_ticket++;
    c->queue.push_back({*ticket, *frame, workspace_bytes(frame, 1, false)});
    serve_progress(c);
    return FM_OK;
}

fm_status fm_serve_poll(fm_ctx* c, uint64_t ticket, int* done) {
    if (!c || !done) return FM_ERR_INVALID_ARG;
    fm_status st = set_device(c);
    if (st != FM_OK) return st;
    serve_progress(c);
    auto it = c->done.find(ticket);
    if (it == c->done.end()) {
        *done = 0;
        for (auto& q : c->queue)
            if (q.ticket == ticket) return FM_OK;
        for (fm_ctx::Slot* sl : c->slots)
            if (sl->busy)
                for (uint64_t t : sl->tickets)
                    if (t == ticket) return FM_OK;
        return fail(c, FM_ERR_NOT_READY, "unknown ticket %llu", (unsigned long long)ticket);
    }
    if (it->second < 0) {
        c->done.erase(it);
        *done = 1;
        return FM_ERR_CUDA;
    }
    *done = 1;
    c->done.erase(it);
    return FM_OK;
}

}  // extern "C"

/*
 * fastmusic.h -- C ABI of the GB300 (sm_103a) fast-MUSIC angle-of-arrival library.
 *
 * The library implements the hot path of arXiv 1911.07434 ("Ultra-Fast
 * Accurate AoA Estimation via Automotive Massive-MIMO Radar") on one GPU:
 *
 *   X (M x T snapshots) --Eq. 2--> R = X X^H / T
 *     --Alg. 1 / Alg. 2--> sketch C = R Pi (+ t power steps V = orth(C), C = R V)
 *     --> W = pinv(P^H C), rank restriction B = R_c W R_c^H, eig(B)  (Sec. III)
 *     --> U_s (M x K signal subspace)
 *     --Eq. 5 / Eq. 10--> P(theta) = 1 / (||a(theta)||^2 - ||U_s^H a(theta)||^2)
 *     --Eq. 6--> the K largest local maxima of P (AoAs)
 *
 * plus plain full-eigendecomposition MUSIC (Eq. 4-6) as the comparison method.
 *
 * Conventions common to every call:
 *   - Pointers named X, R, U, P, peak_* are DEVICE pointers owned by the caller
 *     (e.g. torch tensors' data_ptr()).  The library never frees them.
 *   - Complex values are complex64: interleaved (re, im) float pairs.
 *     Matrices are row-major; X is M x T with leading dimension ldx (complex
 *     elements), row = antenna (Sec. II-B, Eq. 3).
 *   - Every compute call is asynchronous on `stream` (a cudaStream_t; NULL is
 *     the legacy default stream).  Results are valid after the caller
 *     synchronises that stream.  Shapes are validated on the host before any
 *     launch; an invalid call launches nothing and returns FM_ERR_INVALID_ARG.
 *   - Errors are returned as fm_status; a readable message is available from
 *     fm_last_error(ctx).  No exception crosses the ABI.
 *   - Steering vectors follow the far-field signal model of Sec. II-A for a
 *     linear array with element m at position x_m wavelengths along its axis:
 *       a_m(theta) = exp(j 2 pi x_m sin theta),  m = 0..M-1,
 *     theta measured from broadside, grid theta_i = theta0_deg + i * step_deg.
 *     x_m = d_wl * m for a uniform linear array of spacing d_wl (0.5 = lambda/2),
 *     or any positions (a sparse or cascaded MIMO virtual array) given by
 *     fm_array.pos_wl.
 *   - The Gaussian test matrix Pi of Sec. III-B is drawn from Philox4x32-10
 *     (Salmon et al., SC'11) with key (seed_lo, seed_hi) and counter
 *     (column j, row m, frame_id_lo, frame_id_hi); outputs x0, x1 give
 *     u1 = (x0+1)/2^32, u2 = x1/2^32 and Pi[m,j] = sqrt(-2 ln u1) e^{j 2 pi u2}.
 *     The l sampled columns of Alg. 1 come from a partial Fisher-Yates shuffle
 *     whose draw i uses counter (i, 0xFFFFFFFF, frame_id_lo, frame_id_hi) and
 *     j = i + floor(x0 (M - i) / 2^32); the indices are then sorted.
 */
#ifndef FASTMUSIC_H
#define FASTMUSIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* fm_stream; /* == cudaStream_t */
typedef struct fm_ctx fm_ctx;

typedef enum {
    FM_OK = 0,
    FM_ERR_INVALID_ARG = 1,    /* shape/pointer validation failed; nothing launched */
    FM_ERR_CUDA = 2,           /* a CUDA runtime call failed; see fm_last_error */
    FM_ERR_OOM_BUDGET = 3,     /* the call needs more workspace than the context budget */
    FM_ERR_NO_CONVERGENCE = 4, /* (per-frame status bit) an eigensolve hit its sweep cap */
    FM_ERR_TIMEOUT = 5,        /* a bounded wait expired */
    FM_ERR_NOT_READY = 6       /* serving: ticket unknown or still in flight */
} fm_status;

typedef enum {
    FM_FULL_EIG = 0,        /* standard MUSIC, Eq. 4-6 (not served by fm_run; see fm_spectrum) */
    FM_RAND_SAMPLING = 1,   /* fast MUSIC 1, Sec. III-A, Algorithm 1 */
    FM_RAND_PROJECTION = 2  /* fast MUSIC 2, Sec. III-B, Algorithm 2 */
} fm_method;

/* Operand precision of the two large GEMM-shaped steps, the covariance (Eq. 2)
 * and the scan (Eq. 10), when they run on the tensor cores; the accumulator is
 * FP32 in every mode, and the small solves and the main-lobe scan recompute stay
 * FP32 (double-float where stated).  The sketch products (Alg. 1 / 2, Eq. 11) take
 * TF32 operands in TF32 / BF16 mode and 3 TF32 MMAs per product in FP32 mode (see
 * fm_set_sketch_path).  Where the CUDA-core
 * covariance runs instead (X not 16-byte aligned or ldx odd), it is FP32 in
 * every mode.  BF16 keeps FP32's exponent range, so no per-frame scaling is
 * applied. */
typedef enum {
    FM_PREC_FP32 = 0, /* FP32 products: 3 TF32 MMAs per product (hi*hi + hi*lo + lo*hi) */
    FM_PREC_TF32 = 1, /* TF32 operands (10-bit mantissa), one MMA per product */
    FM_PREC_BF16 = 2  /* BF16 operands (7-bit mantissa), one kind::f16 MMA per 16 elements */
} fm_precision;

/* Array geometry (Sec. II-A): M elements on a line.  pos_wl == NULL: a uniform
 * linear array, x_m = d_wl * m with d_wl in (0, 1] wavelengths (0 => 0.5).
 * pos_wl != NULL: a HOST array of M element positions x_m in wavelengths (any
 * order and spacing, |x_m| <= 4096, all finite; d_wl is then ignored).  The
 * library reads pos_wl during the call that takes the frame (fm_run,
 * fm_run_host, fm_graph_create, fm_workspace_bytes) and copies what it needs
 * into its workspace; a frame given to fm_serve_submit is read when its batch
 * starts, so its positions must stay valid until fm_serve_poll reports it done.
 * Frames whose positions are equal element by element share their steering
 * vectors in the scan. */
typedef struct {
    int M;
    double d_wl;
    const double* pos_wl;
} fm_array;

/* Angle grid (Sec. II-B): theta_i = theta0_deg + i * step_deg, i = 0..L-1. */
typedef struct {
    double theta0_deg;
    double step_deg;
    int L;
} fm_grid;

/* Estimator parameters.  K = number of sources, l = sketch size (the paper's p,
 * K <= l <= min(M, 48)), t = power iterations (Eq. 11; 0..8).  rank_restrict:
 * number of columns of U_s used by the scan, K (0 means K) or l.  prec: an
 * fm_precision.  refine = 1 adds one power step computed in FP32 from the
 * snapshots, V = orth(C), C = X (X^H V) / T (= R V without forming R), before the
 * final Rayleigh-Ritz solve, which then uses H = V^H C for both methods; it
 * wins back the accuracy a TF32 / BF16 covariance loses (fm_run only).  seed
 * keys the Philox stream of Pi / the sampled index set. */
typedef struct {
    int method; /* fm_method */
    int K;
    int l;
    int t;
    int prec; /* fm_precision */
    int rank_restrict;
    int refine;
    int reserved_;
    uint64_t seed;
} fm_params;

/* One radar frame for fm_run.  X: device complex64 M x T (ldx >= T).
 * Outputs (device, caller-owned): P_out[L] pseudo-spectrum (FP32, +inf where the
 * denominator is not positive); P_db_out[L] 10 log10 P (nullable); peak_idx[K]
 * grid indices of the K largest local maxima ordered by P descending (ties:
 * lower index), -1 for missing; peak_deg[K] their angles; n_peaks[1] number
 * found; status[1] (nullable) per-frame status bits (0 = ok, FM_ERR_* values
 * OR-ed as 1 << code). */
typedef struct {
    const void* X;
    int T;
    int64_t ldx;
    fm_array arr;
    fm_grid grid;
    fm_params p;
    uint64_t frame_id;
    float* P_out;
    float* P_db_out;
    int* peak_idx;
    float* peak_deg;
    int* n_peaks;
    int* status;
} fm_frame;

/* ---- context -------------------------------------------------------------
 * fm_create: make a context on CUDA device `device` (made current for the
 * calls of this context).  workspace_budget_bytes caps the device workspace
 * the context may hold (0 = 16 GiB); workspace is allocated lazily, grows on
 * demand and is owned (and freed) by the context.  Not thread-safe: one
 * context per host thread. */
fm_status fm_create(fm_ctx** ctx, size_t workspace_budget_bytes, int device);
fm_status fm_destroy(fm_ctx* ctx);
const char* fm_last_error(const fm_ctx* ctx);
/* Device bytes of workspace fm_run needs for these frames (0 on invalid input). */
size_t fm_workspace_bytes(const fm_frame* frames, int n_frames);

/* ---- the whole hot path ------------------------------------------------------
 * fm_run: for every frame, X -> R -> sketch -> U_s -> P -> peaks (Sec. II-III),
 * asynchronously on `stream`.  Frames may differ in every shape parameter.
 * method must be FM_RAND_SAMPLING or FM_RAND_PROJECTION. */
fm_status fm_run(fm_ctx* ctx, const fm_frame* frames, int n_frames, fm_stream stream);

/* ---- autotuning -------------------------------------------------------------------
 * fm_autotune: run fm_run on these frames with every combination of covariance
 * path and scan path (FM_COV_TC / FM_COV_SIMT each) that they can take, `reps`
 * timed runs each after one untimed run (CUDA events on `stream`; synchronises
 * the stream), and keep the fastest combination in the context (as
 * fm_set_cov_path / fm_set_scan_path would).  Reports the choice and its mean
 * milliseconds per fm_run (pointers nullable).  The frames' outputs hold the
 * last run's results. */
fm_status fm_autotune(fm_ctx* ctx, const fm_frame* frames, int n_frames, fm_stream stream, int reps, int* cov_path,
                      int* scan_path, float* best_ms);

/* ---- CUDA graphs ----------------------------------------------------------------
 * fm_graph_create: prepare fm_run's work for these frames once (validation,
 * workspace of its own within the context's budget, descriptors, tensor maps)
 * and capture the chain's kernel launches into a CUDA graph.  The frame
 * pointers are baked in: each fm_graph_launch runs the whole chain again on the
 * current contents of the same X buffers and writes the same output buffers, so
 * a caller that streams frames refills the X buffers between launches.  One
 * plain run of the chain happens inside fm_graph_create (on a private stream,
 * completed before it returns).  fm_graph_launch is asynchronous on `stream`
 * and adds one graph launch; launches of one graph must not overlap each other
 * (they share its workspace).  fm_graph_destroy waits for the device and frees
 * the graph. */
typedef struct fm_graph fm_graph;
fm_status fm_graph_create(fm_ctx* ctx, const fm_frame* frames, int n_frames, fm_graph** graph);
fm_status fm_graph_launch(fm_graph* graph, fm_stream stream);
fm_status fm_graph_destroy(fm_graph* graph);

/* fm_run_subspace: copy U_s (complex64 M x ncols, row-major) of frame `frame` of
 * the most recent fm_run on this context into U (device), asynchronously on
 * `stream`.  The copy reads the context's workspace, so it must be issued before
 * the next call that uses this context; FM_ERR_INVALID_ARG if there is no such
 * frame. */
fm_status fm_run_subspace(fm_ctx* ctx, int frame, void* U, fm_stream stream);

/* fm_run_host: fm_run for frames whose X and outputs are in host memory
 * (page-locked memory lets the copies run asynchronously; pageable memory works
 * but the copies then block the host).  Asynchronous: the call enqueues, on
 * streams of the context, the host -> device copies of every X (rows of T
 * complex elements taken with stride ldx) into one of two device staging
 * slots (frames adjacent in host memory in one copy), the whole chain, and the
 * device -> host transfer of every output, and makes `stream` wait for it, so
 * once `stream` has passed the call the host outputs are written.  Where the
 * device addresses host memory through host pointers
 * (cudaDevAttrPageableMemoryAccess) and every output is 4-byte aligned, one
 * kernel writes all outputs into the host buffers; otherwise each output buffer
 * is copied (one cudaMemcpyAsync each).  The two staging slots alternate, so a call
 * may block the host until the call two before it has written its outputs.
 * Consecutive calls overlap: the copies of one
 * call run while the previous call computes.  The host X must hold its data
 * when the call is made (the copies in do not wait for earlier work on
 * `stream`), and the caller keeps the host buffers of a call untouched until
 * `stream` has passed it.  The staging slots are
 * device memory of the context outside the workspace budget (the frames' X and
 * outputs, twice). */
fm_status fm_run_host(fm_ctx* ctx, const fm_frame* frames, int n_frames, fm_stream stream);

/* fm_selftest_wait_timeout: self-test of failure detection (the paper has no
 * counterpart).  Launches one warp that waits, with the bounded mbarrier wait of
 * the tensor-core kernels, on a barrier that nothing arrives on; after limit_ms
 * (converted to SM clocks at the device's maximum clock) the wait gives up, the
 * kernel ORs the FM_ERR_TIMEOUT bit (1 << FM_ERR_TIMEOUT) into *status (device
 * int) and returns normally, so the context stays usable.  limit_ms in (0, 1e4]. */
fm_status fm_selftest_wait_timeout(fm_ctx* ctx, int* status, double limit_ms, fm_stream stream);

/* ---- steps (uniform batches; each frame at a fixed stride) ------------------
 * fm_covariance (Eq. 2): R_b = X_b X_b^H / T for b < n_frames.  X_b = X +
 * b * x_frame_stride complex elements; R_b = R + b*M*M (complex64, full
 * Hermitian matrix written).  prec: an fm_precision (tensor-core path only). */
fm_status fm_covariance(fm_ctx* ctx, const void* X, int n_frames, int M, int T, int64_t ldx,
                        int64_t x_frame_stride, void* R, int prec, fm_stream stream);

/* fm_subspace (Alg. 1 / Alg. 2): randomized signal subspace of each R_b
 * (complex64 M x M at R + b*M*M).  U_b = U + b*M*ncols (complex64, M x ncols,
 * ncols = p->rank_restrict or K); frame b uses frame_id0 + b for its Philox
 * stream.  status[b] (nullable) receives the per-frame status bits. */
fm_status fm_subspace(fm_ctx* ctx, const void* R, int n_frames, int M, const fm_params* p,
                      uint64_t frame_id0, void* U, int* status, fm_stream stream);

/* fm_spectrum (Eq. 5 / Eq. 10): P_b[i] = 1/(M - ||U_b^H a(theta_i)||^2) for
 * U_b = U + b*M*ncols (complex64 M x ncols, orthonormal columns), P_b = P + b*L,
 * on a uniform linear array of spacing d_wl. */
fm_status fm_spectrum(fm_ctx* ctx, const void* U, int n_frames, int M, int ncols, double d_wl,
                      const fm_grid* grid, float* P, fm_stream stream);
/* fm_spectrum_array: fm_spectrum for the array `arr` (uniform or given by
 * arr->pos_wl, read during the call); M = arr->M. */
fm_status fm_spectrum_array(fm_ctx* ctx, const void* U, int n_frames, const fm_array* arr, int ncols,
                            const fm_grid* grid, float* P, fm_stream stream);

/* fm_peaks (Eq. 6): K largest local maxima of each P_b (P + b*L); a local
 * maximum is i with P[i] > P[i-1] and P[i] >= P[i+1] (missing neighbours at the
 * ends never block).  Outputs at peak_idx + b*K, peak_deg + b*K, n_peaks + b. */
fm_status fm_peaks(fm_ctx* ctx, const float* P, int n_frames, int L, int K, const fm_grid* grid,
                   int* peak_idx, float* peak_deg, int* n_peaks, fm_stream stream);

/* fm_test_matrix: the Gaussian Pi (complex64 M x l, row-major) of frame_id. */
fm_status fm_test_matrix(fm_ctx* ctx, uint64_t seed, uint64_t frame_id, int M, int l, void* Pi,
                         fm_stream stream);
/* fm_sample_indices: the sorted index set I (l int32) of Algorithm 1. */
fm_status fm_sample_indices(fm_ctx* ctx, uint64_t seed, uint64_t frame_id, int M, int l, int* idx,
                            fm_stream stream);

/* ---- per-stage timing (CUDA events on the launching stream) -----------------
 * When enabled, every stage launch inside fm_run / step calls is bracketed by
 * events.  fm_stage_times synchronises on them and returns, per stage, the
 * summed milliseconds and the number of launches since the last reset.
 * Stage order: 0 grid table, 1 covariance, 2 sketch, 3 orth, 4 final small
 * solve, 5 scan, 6 peaks, 7 FP32 refinement step.  fm_set_timing(ctx, 1) times
 * every stage, 0 none; fm_set_timing_mask times the stages whose bit
 * (1 << stage) is set in mask (each timed launch adds two event records to its
 * stream, so timing one stage perturbs a step less than timing all of them). */
#define FM_N_STAGES 8
fm_status fm_set_timing(fm_ctx* ctx, int enable);
fm_status fm_set_timing_mask(fm_ctx* ctx, unsigned mask);
fm_status fm_stage_times(fm_ctx* ctx, double* total_ms, int* launches, int reset);
/* Number of kernel launches issued by this context since creation. */
uint64_t fm_launch_count(const fm_ctx* ctx);

/* ---- covariance kernel selection ----------------------------------------------
 * FM_COV_AUTO (default): the tensor-core kernel (tcgen05 MMAs with TMEM
 * accumulators, TMA-staged tiles, FP32-level accuracy from three TF32 products
 * per FP32 product) whenever every frame's X is 16-byte aligned with an even
 * ldx, else the FP32 CUDA-core kernel.  FM_COV_SIMT / FM_COV_TC force one path
 * (FM_COV_TC fails with FM_ERR_INVALID_ARG for frames it cannot take).
 * fm_last_cov_path returns the path the latest covariance launch used. */
#define FM_COV_AUTO 0
#define FM_COV_SIMT 1
#define FM_COV_TC 2
fm_status fm_set_cov_path(fm_ctx* ctx, int path);
int fm_last_cov_path(const fm_ctx* ctx);

/* ---- scan kernel selection (same constants) -------------------------------------
 * Inside fm_run the frames are grouped by (M, number of U_s columns, angle
 * grid, prec).  A group on the tensor cores is scanned by one batched launch
 * (the steering tile generated in registers serves every frame of the group;
 * tcgen05 MMAs, 3 TF32 products per FP32 product in FP32 mode), after which the
 * angles of the main lobes (||U_s^H a||^2 above 4 times the number of U_s
 * columns, where M - ||U_s^H a||^2 cancels) are recomputed by the FP32
 * CUDA-core scan.  FM_COV_AUTO (default): the tensor cores take the groups
 * whose frames fill at least a quarter of the kernel's B tile (frames >=
 * 64 / ncols rounded up to a power of two), the CUDA-core scan the rest;
 * FM_COV_TC: every group on the tensor cores; FM_COV_SIMT: the CUDA-core scan
 * for every frame.  fm_last_scan_path reports FM_COV_TC or FM_COV_SIMT when
 * all frames of the last fm_run took that path, FM_COV_AUTO when both ran.
 * fm_spectrum always uses the CUDA-core scan. */
fm_status fm_set_scan_path(fm_ctx* ctx, int path);
int fm_last_scan_path(const fm_ctx* ctx);

/* ---- sketch kernel selection (same constants) -----------------------------------
 * The sketch products C = R Omega (Alg. 2) and C = R V of the power steps (Eq. 11)
 * run on the tensor cores for every frame whose M is even (R's rows must be
 * 16-byte aligned for TMA): every product of an FP32 frame with 3 TF32 MMAs per
 * FP32 product (hi*hi + hi*lo + lo*hi), those of TF32 / BF16 frames with one.  The
 * sampling sketch of Alg. 1 (a column gather) is not a product.  FM_COV_AUTO
 * (default): the tensor cores take the frames that can; FM_COV_TC: the same, and
 * fm_run fails with FM_ERR_INVALID_ARG if a frame with a product cannot;
 * FM_COV_SIMT: every product on the FP32 CUDA cores.  fm_last_sketch_path reports
 * FM_COV_TC or FM_COV_SIMT when every frame with a product took that path,
 * FM_COV_AUTO when both ran.  fm_subspace always uses the CUDA cores. */
fm_status fm_set_sketch_path(fm_ctx* ctx, int path);
int fm_last_sketch_path(const fm_ctx* ctx);

/* ---- eigensolver sweep cap (failure detection) -----------------------------------
 * The paper's SVD / eigendecomposition steps (Alg. 1 / Alg. 2) run here as cyclic
 * Jacobi iterations on l x l matrices with a cap of 30 sweeps; a frame whose
 * solve does not converge within the cap (or meets a non-finite pivot) still
 * gets outputs, and its status word carries the FM_ERR_NO_CONVERGENCE bit.
 * fm_set_sweep_cap lowers the cap for the later fm_run calls of this context
 * (and for the graphs and serving slots created after it): cap in [1, 30], 0
 * restores 30.  A cap of 1 makes an ordinary frame report FM_ERR_NO_CONVERGENCE,
 * which is how failure detection is exercised without faulting anything. */
fm_status fm_set_sweep_cap(fm_ctx* ctx, int cap);

/* ---- allocation-free spectrum --------------------------------------------------
 * The paper has no counterpart to this call; it exists for callers that cannot
 * let the library allocate device memory: a radar front end that fixes its
 * memory map at start-up and must not allocate while frames stream in, or a host
 * framework that owns every device allocation itself.  fm_spectrum_noalloc
 * computes exactly what fm_spectrum computes (same kernels, same results) but
 * takes no context and allocates nothing: its scratch (frame descriptors and
 * the steering-phase table of the grid) lives in a fixed array inside the
 * library, about 524 KB, which every GPU that loads the library holds until the
 * process exits.  Limits: n_frames <= 64 and grid->L <= 65536 (larger requests
 * return FM_ERR_INVALID_ARG before any work), plus fm_spectrum's own limits.
 * Every call looks up the array's device address on the current device
 * (cudaGetSymbolAddress, which also loads the module there on the first call of
 * a process), so a device reset between calls is harmless; make the first call
 * on a device before any stream capture.  Every call shares the one array and overwrites it: calls that
 * overlap on the GPU (different streams, or different host threads on one
 * device) race, so serialise them on one stream.  The descriptors are copied
 * from host stack memory with a pageable cudaMemcpyAsync, which has taken its
 * own copy of them when it returns.  Returns FM_OK, FM_ERR_INVALID_ARG or
 * FM_ERR_CUDA (there is no context, hence no fm_last_error text). */
fm_status fm_spectrum_noalloc(const void* U, int n_frames, int M, int ncols, double d_wl, const fm_grid* grid,
                              float* P, fm_stream stream);

/* ---- serving (continuous batching) ------------------------------------------
 * fm_serve_submit: enqueue one frame (validated as in fm_run; a frame whose
 * workspace alone exceeds the context budget returns FM_ERR_OOM_BUDGET) and set
 * *ticket.  The library runs up to 4 slots, each a stream with a private
 * workspace.  Whenever a slot is free it takes the queued frames in arrival
 * order, up to 64 and as many as the budget left beside the other slots'
 * workspaces allows, and runs them as one fm_run batch; frames that arrive
 * while others run overlap with them on the GPU, and under load the batches
 * grow.  Queued work advances inside fm_serve_submit and fm_serve_poll.
 * fm_serve_poll sets *done = 1 once the frame's outputs are complete on the
 * device (FM_ERR_CUDA with *done = 1 if its batch failed; FM_ERR_NOT_READY for
 * an unknown ticket).  The caller's X and output buffers must stay valid until
 * then.  A frame's result does not depend on its batch beyond rounding: the
 * scan groups of a batch, hence the order of the tensor-core accumulation,
 * depend on the batch, within the scan tolerance. */
fm_status fm_serve_submit(fm_ctx* ctx, const fm_frame* frame, uint64_t* ticket);
fm_status fm_serve_poll(fm_ctx* ctx, uint64_t ticket, int* done);

#ifdef __cplusplus
}
#endif

#endif /* FASTMUSIC_H */

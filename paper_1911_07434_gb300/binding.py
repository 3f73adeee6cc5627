"""Thin ctypes binding of the C ABI in include/fastmusic.h (argument marshalling only).

Every computation runs in libfastmusic.so (CUDA, sm_103a).  There is no CPU or
PyTorch fallback: if the library has not been built, `load()` raises.  Build it
with `paper_1911_07434_gb300.build.build()` (or `__graft_entry__.build()`).

The module-level functions carry the C names (fm_create, fm_run, ...) and take
raw pointers; `Context` wraps them for torch tensors (device memory and the
current CUDA stream come from PyTorch).
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, byref, c_double, c_float, c_int, c_int64, c_size_t, c_uint, c_uint64, c_void_p

from . import build as _build

FM_OK = 0
FM_ERR_INVALID_ARG = 1
FM_ERR_CUDA = 2
FM_ERR_OOM_BUDGET = 3
FM_ERR_NO_CONVERGENCE = 4
FM_ERR_TIMEOUT = 5
FM_ERR_NOT_READY = 6

FM_FULL_EIG = 0
FM_RAND_SAMPLING = 1
FM_RAND_PROJECTION = 2

FM_PREC_FP32 = 0
FM_PREC_TF32 = 1
FM_PREC_BF16 = 2
FM_COV_AUTO = 0
FM_COV_SIMT = 1
FM_COV_TC = 2
FM_N_STAGES = 8
STAGES = ("grid", "covariance", "sketch", "orth", "final", "scan", "peaks", "refine")


class FmArray(ctypes.Structure):
    _fields_ = [("M", c_int), ("d_wl", c_double), ("pos_wl", c_void_p)]


class FmGrid(ctypes.Structure):
    _fields_ = [("theta0_deg", c_double), ("step_deg", c_double), ("L", c_int)]


class FmParams(ctypes.Structure):
    _fields_ = [("method", c_int), ("K", c_int), ("l", c_int), ("t", c_int), ("prec", c_int),
                ("rank_restrict", c_int), ("refine", c_int), ("reserved_", c_int), ("seed", c_uint64)]


class FmFrame(ctypes.Structure):
    _fields_ = [("X", c_void_p), ("T", c_int), ("ldx", c_int64), ("arr", FmArray), ("grid", FmGrid),
                ("p", FmParams), ("frame_id", c_uint64), ("P_out", c_void_p), ("P_db_out", c_void_p),
                ("peak_idx", c_void_p), ("peak_deg", c_void_p), ("n_peaks", c_void_p), ("status", c_void_p)]


_lib = None

_SIGS = {
    "fm_create": (c_int, [POINTER(c_void_p), c_size_t, c_int]),
    "fm_destroy": (c_int, [c_void_p]),
    "fm_last_error": (ctypes.c_char_p, [c_void_p]),
    "fm_workspace_bytes": (c_size_t, [POINTER(FmFrame), c_int]),
    "fm_run": (c_int, [c_void_p, POINTER(FmFrame), c_int, c_void_p]),
    "fm_covariance": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_int64, c_int64, c_void_p, c_int, c_void_p]),
    "fm_subspace": (c_int, [c_void_p, c_void_p, c_int, c_int, POINTER(FmParams), c_uint64, c_void_p, c_void_p,
                            c_void_p]),
    "fm_spectrum": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_double, POINTER(FmGrid), c_void_p, c_void_p]),
    "fm_spectrum_array": (c_int, [c_void_p, c_void_p, c_int, POINTER(FmArray), c_int, POINTER(FmGrid), c_void_p,
                                  c_void_p]),
    "fm_peaks": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, POINTER(FmGrid), c_void_p, c_void_p, c_void_p,
                         c_void_p]),
    "fm_test_matrix": (c_int, [c_void_p, c_uint64, c_uint64, c_int, c_int, c_void_p, c_void_p]),
    "fm_sample_indices": (c_int, [c_void_p, c_uint64, c_uint64, c_int, c_int, c_void_p, c_void_p]),
    "fm_set_timing": (c_int, [c_void_p, c_int]),
    "fm_set_timing_mask": (c_int, [c_void_p, c_uint]),
    "fm_stage_times": (c_int, [c_void_p, POINTER(c_double), POINTER(c_int), c_int]),
    "fm_launch_count": (c_uint64, [c_void_p]),
    "fm_run_subspace": (c_int, [c_void_p, c_int, c_void_p, c_void_p]),
    "fm_run_host": (c_int, [c_void_p, POINTER(FmFrame), c_int, c_void_p]),
    "fm_selftest_wait_timeout": (c_int, [c_void_p, c_void_p, c_double, c_void_p]),
    "fm_autotune": (c_int, [c_void_p, POINTER(FmFrame), c_int, c_void_p, c_int, POINTER(c_int), POINTER(c_int),
                            POINTER(c_float)]),
    "fm_graph_create": (c_int, [c_void_p, POINTER(FmFrame), c_int, POINTER(c_void_p)]),
    "fm_graph_launch": (c_int, [c_void_p, c_void_p]),
    "fm_graph_destroy": (c_int, [c_void_p]),
    "fm_set_cov_path": (c_int, [c_void_p, c_int]),
    "fm_last_cov_path": (c_int, [c_void_p]),
    "fm_set_scan_path": (c_int, [c_void_p, c_int]),
    "fm_last_scan_path": (c_int, [c_void_p]),
    "fm_set_sketch_path": (c_int, [c_void_p, c_int]),
    "fm_last_sketch_path": (c_int, [c_void_p]),
    "fm_set_sweep_cap": (c_int, [c_void_p, c_int]),
    "fm_spectrum_noalloc": (c_int, [c_void_p, c_int, c_int, c_int, c_double, POINTER(FmGrid), c_void_p, c_void_p]),
    "fm_serve_submit": (c_int, [c_void_p, POINTER(FmFrame), POINTER(c_uint64)]),
    "fm_serve_poll": (c_int, [c_void_p, c_uint64, POINTER(c_int)]),
}


def library_path() -> str:
    return _build.LIB


def load():
    """Load libfastmusic.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"CUDA library {path} is missing: build it with paper_1911_07434_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return list(_SIGS.keys())


# ---- C names, raw pointers --------------------------------------------------
def fm_create(budget_bytes: int = 0, device: int = 0) -> int:
    h = c_void_p()
    st = load().fm_create(byref(h), budget_bytes, device)
    if st != FM_OK:
        raise RuntimeError(f"fm_create failed with status {st}")
    return h.value


def fm_destroy(ctx: int) -> int:
    return load().fm_destroy(ctx)


def fm_last_error(ctx: int) -> str:
    r = load().fm_last_error(ctx)
    return r.decode() if r else ""


def fm_workspace_bytes(frames) -> int:
    arr = (FmFrame * len(frames))(*frames)
    return load().fm_workspace_bytes(arr, len(frames))


def fm_run(ctx, frames, stream) -> int:
    arr = (FmFrame * len(frames))(*frames)
    return load().fm_run(ctx, arr, len(frames), stream)


def fm_covariance(ctx, X, n_frames, M, T, ldx, x_frame_stride, R, prec, stream) -> int:
    return load().fm_covariance(ctx, X, n_frames, M, T, ldx, x_frame_stride, R, prec, stream)


def fm_subspace(ctx, R, n_frames, M, params: FmParams, frame_id0, U, status, stream) -> int:
    return load().fm_subspace(ctx, R, n_frames, M, byref(params), frame_id0, U, status, stream)


def fm_spectrum(ctx, U, n_frames, M, ncols, d_wl, grid: FmGrid, P, stream) -> int:
    return load().fm_spectrum(ctx, U, n_frames, M, ncols, d_wl, byref(grid), P, stream)


def fm_spectrum_array(ctx, U, n_frames, arr: FmArray, ncols, grid: FmGrid, P, stream) -> int:
    return load().fm_spectrum_array(ctx, U, n_frames, byref(arr), ncols, byref(grid), P, stream)


def fm_peaks(ctx, P, n_frames, L, K, grid: FmGrid, peak_idx, peak_deg, n_peaks, stream) -> int:
    return load().fm_peaks(ctx, P, n_frames, L, K, byref(grid), peak_idx, peak_deg, n_peaks, stream)


def fm_test_matrix(ctx, seed, frame_id, M, l, Pi, stream) -> int:
    return load().fm_test_matrix(ctx, seed, frame_id, M, l, Pi, stream)


def fm_sample_indices(ctx, seed, frame_id, M, l, idx, stream) -> int:
    return load().fm_sample_indices(ctx, seed, frame_id, M, l, idx, stream)


def fm_set_timing(ctx, enable) -> int:
    return load().fm_set_timing(ctx, int(enable))


def fm_set_timing_mask(ctx, mask) -> int:
    return load().fm_set_timing_mask(ctx, int(mask))


def fm_stage_times(ctx, reset=False):
    ms = (c_double * FM_N_STAGES)()
    n = (c_int * FM_N_STAGES)()
    st = load().fm_stage_times(ctx, ms, n, int(reset))
    return st, list(ms), list(n)


def fm_autotune(ctx, frames, stream, reps):
    arr = (FmFrame * len(frames))(*frames)
    cp, sp, ms = c_int(), c_int(), c_float()
    st = load().fm_autotune(ctx, arr, len(frames), stream, reps, byref(cp), byref(sp), byref(ms))
    return st, cp.value, sp.value, ms.value


def fm_graph_create(ctx, frames):
    arr = (FmFrame * len(frames))(*frames)
    g = c_void_p()
    st = load().fm_graph_create(ctx, arr, len(frames), byref(g))
    return st, g.value


def fm_graph_launch(graph, stream) -> int:
    return load().fm_graph_launch(graph, stream)


def fm_graph_destroy(graph) -> int:
    return load().fm_graph_destroy(graph)


def fm_selftest_wait_timeout(ctx, status, limit_ms, stream) -> int:
    return load().fm_selftest_wait_timeout(ctx, status, limit_ms, stream)


def fm_run_host(ctx, frames, stream) -> int:
    arr = (FmFrame * len(frames))(*frames)
    return load().fm_run_host(ctx, arr, len(frames), stream)


def fm_run_subspace(ctx, frame, U, stream) -> int:
    return load().fm_run_subspace(ctx, frame, U, stream)


def fm_launch_count(ctx) -> int:
    return load().fm_launch_count(ctx)


def fm_set_cov_path(ctx, path) -> int:
    return load().fm_set_cov_path(ctx, path)


def fm_last_cov_path(ctx) -> int:
    return load().fm_last_cov_path(ctx)


def fm_set_scan_path(ctx, path) -> int:
    return load().fm_set_scan_path(ctx, path)


def fm_last_scan_path(ctx) -> int:
    return load().fm_last_scan_path(ctx)


def fm_set_sketch_path(ctx, path) -> int:
    return load().fm_set_sketch_path(ctx, path)


def fm_last_sketch_path(ctx) -> int:
    return load().fm_last_sketch_path(ctx)


def fm_set_sweep_cap(ctx, cap) -> int:
    return load().fm_set_sweep_cap(ctx, cap)


def fm_spectrum_noalloc(U, n_frames, M, ncols, d_wl, grid: FmGrid, P, stream) -> int:
    """Same result as fm_spectrum without any device allocation (see fastmusic.h)."""
    return load().fm_spectrum_noalloc(U, n_frames, M, ncols, d_wl, byref(grid), P, stream)


def fm_serve_submit(ctx, frame: FmFrame):
    t = c_uint64()
    st = load().fm_serve_submit(ctx, byref(frame), byref(t))
    return st, t.value


def fm_serve_poll(ctx, ticket):
    d = c_int()
    st = load().fm_serve_poll(ctx, ticket, byref(d))
    return st, d.value


# ---- torch convenience ------------------------------------------------------
def _array(M, d_wl, pos_wl, owner) -> FmArray:
    """FmArray of M elements; with positions, a float64 copy is kept alive on `owner`."""
    if pos_wl is None:
        return FmArray(M, d_wl, None)
    import numpy as np
    pos = np.ascontiguousarray(pos_wl, dtype=np.float64)
    if pos.shape != (M,):
        raise ValueError(f"pos_wl must hold M = {M} positions")
    owner._pos_keep = pos
    return FmArray(M, d_wl, pos.ctypes.data)



def _stream_handle(stream=None) -> int:
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


class FmError(RuntimeError):
    pass


class Context:
    """Owns an fm_ctx; methods take torch CUDA tensors and run on the current stream."""

    def __init__(self, budget_bytes: int = 0, device: int = 0):
        self.device = device
        self.h = fm_create(budget_bytes, device)

    def close(self):
        if self.h:
            fm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st != FM_OK:
            raise FmError(f"{what}: status {st}: {fm_last_error(self.h)}")

    # frames -----------------------------------------------------------------
    @staticmethod
    def frame(X, K, l, t, method, theta0, step, L, P, peak_idx, peak_deg, n_peaks, seed=0, frame_id=0,
              d_wl=0.5, status=None, P_db=None, rank_restrict=0, prec=0, refine=0, pos_wl=None) -> FmFrame:
        """FmFrame for a complex64 CUDA tensor X (M x T, row stride >= T).  pos_wl: element
        positions in wavelengths (M floats; None = uniform spacing d_wl); the frame keeps
        a float64 copy alive for the library to read."""
        M, T = X.shape
        f = FmFrame()
        f.X = X.data_ptr()
        f.T = T
        f.ldx = X.stride(0)
        f.arr = _array(M, d_wl, pos_wl, f)
        f.grid = FmGrid(theta0, step, L)
        f.p = FmParams(method, K, l, t, prec, rank_restrict, refine, 0, seed)
        f.frame_id = frame_id
        f.P_out = P.data_ptr()
        f.P_db_out = P_db.data_ptr() if P_db is not None else None
        f.peak_idx = peak_idx.data_ptr()
        f.peak_deg = peak_deg.data_ptr()
        f.n_peaks = n_peaks.data_ptr()
        f.status = status.data_ptr() if status is not None else None
        return f

    def run_host(self, frames, stream=None):
        """fm_run on frames whose X and outputs are host (pinned) tensors; asynchronous."""
        self._check(fm_run_host(self.h, frames, _stream_handle(stream)), "fm_run_host")

    def run(self, frames, stream=None):
        self._check(fm_run(self.h, frames, _stream_handle(stream)), "fm_run")

    def autotune(self, frames, reps=3, stream=None):
        """Pick the fastest covariance / scan paths for these frames; returns (cov, scan, ms)."""
        st, cp, sp, ms = fm_autotune(self.h, frames, _stream_handle(stream), reps)
        self._check(st, "fm_autotune")
        return cp, sp, ms

    def graph(self, frames):
        """CUDA graph of the whole chain for these frames (see fm_graph_create)."""
        st, g = fm_graph_create(self.h, frames)
        self._check(st, "fm_graph_create")
        return Graph(self, g)

    def run_subspace(self, frame: int, M: int, ncols: int, stream=None):
        """U_s (M x ncols complex64) of frame `frame` of the last run() on this context."""
        import torch
        U = torch.empty((M, ncols), dtype=torch.complex64, device=f"cuda:{self.device}")
        self._check(fm_run_subspace(self.h, frame, U.data_ptr(), _stream_handle(stream)), "fm_run_subspace")
        return U

    def covariance(self, X, R=None, stream=None, prec=FM_PREC_FP32):
        """X: (B, M, T) or (M, T) complex64 CUDA tensor -> R (B, M, M) complex64."""
        import torch
        Xb = X if X.dim() == 3 else X.unsqueeze(0)
        B, M, T = Xb.shape
        assert Xb.stride(2) == 1
        if R is None:
            R = torch.empty((B, M, M), dtype=torch.complex64, device=X.device)
        self._check(fm_covariance(self.h, Xb.data_ptr(), B, M, T, Xb.stride(1), Xb.stride(0), R.data_ptr(),
                                  prec, _stream_handle(stream)), "fm_covariance")
        return R

    def subspace(self, R, K, l, t, method, seed=0, frame_id0=0, rank_restrict=0, stream=None):
        import torch
        Rb = R if R.dim() == 3 else R.unsqueeze(0)
        B, M, _ = Rb.shape
        Rb = Rb.contiguous()
        nc = l if rank_restrict == l else K
        U = torch.empty((B, M, nc), dtype=torch.complex64, device=R.device)
        status = torch.zeros(B, dtype=torch.int32, device=R.device)
        p = FmParams(method, K, l, t, FM_PREC_FP32, rank_restrict, 0, 0, seed)
        self._check(fm_subspace(self.h, Rb.data_ptr(), B, M, p, frame_id0, U.data_ptr(), status.data_ptr(),
                                _stream_handle(stream)), "fm_subspace")
        return U, status

    def spectrum(self, U, theta0, step, L, d_wl=0.5, stream=None):
        import torch
        Ub = (U if U.dim() == 3 else U.unsqueeze(0)).contiguous()
        B, M, nc = Ub.shape
        P = torch.empty((B, L), dtype=torch.float32, device=U.device)
        self._check(fm_spectrum(self.h, Ub.data_ptr(), B, M, nc, d_wl, FmGrid(theta0, step, L), P.data_ptr(),
                                _stream_handle(stream)), "fm_spectrum")
        return P

    def spectrum_array(self, U, theta0, step, L, pos_wl=None, d_wl=0.5, stream=None):
        """fm_spectrum_array: the scan for element positions pos_wl (None: uniform d_wl)."""
        import torch
        Ub = (U if U.dim() == 3 else U.unsqueeze(0)).contiguous()
        B, M, nc = Ub.shape
        P = torch.empty((B, L), dtype=torch.float32, device=U.device)
        arr = _array(M, d_wl, pos_wl, self)
        self._check(fm_spectrum_array(self.h, Ub.data_ptr(), B, arr, nc, FmGrid(theta0, step, L), P.data_ptr(),
                                      _stream_handle(stream)), "fm_spectrum_array")
        return P

    def set_sweep_cap(self, cap: int):
        """Jacobi sweeps allowed in the l x l eigensolves of later runs (0: the default 30)."""
        self._check(fm_set_sweep_cap(self.h, cap), "fm_set_sweep_cap")

    def peaks(self, P, K, theta0, step, stream=None):
        import torch
        Pb = (P if P.dim() == 2 else P.unsqueeze(0)).contiguous()
        B, L = Pb.shape
        idx = torch.empty((B, K), dtype=torch.int32, device=P.device)
        deg = torch.empty((B, K), dtype=torch.float32, device=P.device)
        n = torch.empty(B, dtype=torch.int32, device=P.device)
        self._check(fm_peaks(self.h, Pb.data_ptr(), B, L, K, FmGrid(theta0, step, L), idx.data_ptr(),
                             deg.data_ptr(), n.data_ptr(), _stream_handle(stream)), "fm_peaks")
        return idx, deg, n

    def test_matrix(self, seed, frame_id, M, l, stream=None):
        import torch
        out = torch.empty((M, l), dtype=torch.complex64, device=f"cuda:{self.device}")
        self._check(fm_test_matrix(self.h, seed, frame_id, M, l, out.data_ptr(), _stream_handle(stream)),
                    "fm_test_matrix")
        return out

    def sample_indices(self, seed, frame_id, M, l, stream=None):
        import torch
        out = torch.empty(l, dtype=torch.int32, device=f"cuda:{self.device}")
        self._check(fm_sample_indices(self.h, seed, frame_id, M, l, out.data_ptr(), _stream_handle(stream)),
                    "fm_sample_indices")
        return out

    def set_timing(self, on: bool):
        self._check(fm_set_timing(self.h, on), "fm_set_timing")

    def set_timing_mask(self, mask: int):
        """Time only the stages whose bit (1 << stage) is set."""
        self._check(fm_set_timing_mask(self.h, mask), "fm_set_timing_mask")

    def stage_times(self, reset=False):
        st, ms, n = fm_stage_times(self.h, reset)
        self._check(st, "fm_stage_times")
        return {name: (ms[i], n[i]) for i, name in enumerate(STAGES)}

    def launch_count(self) -> int:
        return fm_launch_count(self.h)

    def set_cov_path(self, path: int):
        self._check(fm_set_cov_path(self.h, path), "fm_set_cov_path")

    def last_cov_path(self) -> int:
        return fm_last_cov_path(self.h)

    def set_scan_path(self, path: int):
        self._check(fm_set_scan_path(self.h, path), "fm_set_scan_path")

    def last_scan_path(self) -> int:
        return fm_last_scan_path(self.h)

    def set_sketch_path(self, path: int):
        self._check(fm_set_sketch_path(self.h, path), "fm_set_sketch_path")

    def last_sketch_path(self) -> int:
        return fm_last_sketch_path(self.h)

    def serve_submit(self, frame: FmFrame) -> int:
        st, t = fm_serve_submit(self.h, frame)
        self._check(st, "fm_serve_submit")
        return t

    def serve_poll(self, ticket: int) -> bool:
        st, d = fm_serve_poll(self.h, ticket)
        self._check(st, "fm_serve_poll")
        return bool(d)


class Graph:
    """A captured fm_run chain; launch() re-runs it on the frames' current inputs."""

    def __init__(self, ctx: Context, handle):
        self.ctx = ctx
        self.h = handle

    def launch(self, stream=None):
        self.ctx._check(fm_graph_launch(self.h, _stream_handle(stream)), "fm_graph_launch")

    def close(self):
        if self.h:
            fm_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

"""FP64 CPU oracle for the fast-MUSIC path (arXiv 1911.07434) -- TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline /
reference leg may import this package.  The CUDA library never does, and this
package never loads the CUDA library.  The arithmetic lives in
``fastmusic_oracle.c`` (plain C99, double complex); this module only compiles it
with gcc and marshals numpy arrays through ctypes.

Function map (paper section / equation / algorithm each one follows):
  covariance          Eq. 2              S = Y Y^H / N
  eigh_jacobi         Eq. 4              cyclic complex Jacobi EVD of a Hermitian matrix
  svd_jacobi          Alg. 1 (SVD of C)  one-sided Jacobi thin SVD
  householder_qr      Sec. III-B qr()/orth()
  pinv_hermitian      Eq. 8              pseudo-inverse by EVD
  philox4x32_10       counter-based generator used for Pi (Salmon et al., SC'11)
  gaussian_test_matrix Sec. III-B        complex Gaussian Pi
  sample_indices      Alg. 1             index set I
  music_subspace      Eq. 4              U_K of standard MUSIC
  fast_music          Alg. 1 / Alg. 2    randomized signal subspace
  spectrum            Eq. 5 / Eq. 10     pseudo-spectrum on an angle grid (uniform or given positions)
  peaks               Eq. 6              K largest local maxima
  frame               whole frame X -> P, peaks
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fastmusic_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

SAMPLING = 1
PROJECTION = 2
FULL_EIG = 0


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        c_int, c_u64, c_dbl, c_i64 = ctypes.c_int, ctypes.c_uint64, ctypes.c_double, ctypes.c_int64
        vp = ctypes.c_void_p
        sig = {
            "orc_philox4x32_10": (None, [vp, vp, vp]),
            "orc_gaussian_test_matrix": (None, [c_u64, c_u64, c_int, c_int, vp]),
            "orc_sample_indices": (c_int, [c_u64, c_u64, c_int, c_int, vp]),
            "orc_covariance": (c_int, [vp, c_int, c_int, c_i64, vp]),
            "orc_eigh_jacobi": (c_int, [c_int, vp, vp, vp, c_dbl, c_int]),
            "orc_svd_jacobi": (c_int, [c_int, c_int, vp, vp, vp, vp, c_dbl, c_int]),
            "orc_householder_qr": (c_int, [c_int, c_int, vp, vp, vp]),
            "orc_pinv_hermitian": (c_int, [c_int, vp, vp]),
            "orc_music_subspace": (c_int, [vp, c_int, c_int, vp, vp]),
            "orc_fast_music": (c_int, [vp, c_int, c_int, c_int, c_int, c_int, c_u64, c_u64,
                                       c_int, c_int, vp, vp, vp]),
            "orc_spectrum": (c_int, [vp, c_int, c_int, c_dbl, vp, c_dbl, c_dbl, c_int, c_int, vp]),
            "orc_peaks": (c_int, [vp, c_int, c_int, vp, vp]),
            "orc_frame": (c_int, [vp, c_int, c_int, c_i64, c_int, c_int, c_int, c_int, c_u64,
                                  c_u64, c_dbl, vp, c_dbl, c_dbl, c_int, vp, vp, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc: int, what: str) -> int:
    if rc < 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")
    return rc


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def gaussian_test_matrix(seed: int, frame_id: int, M: int, l: int) -> np.ndarray:
    out = np.zeros((M, l), dtype=np.complex128)
    _load().orc_gaussian_test_matrix(seed, frame_id, M, l, _p(out))
    return out


def sample_indices(seed: int, frame_id: int, M: int, l: int) -> np.ndarray:
    out = np.zeros(l, dtype=np.int32)
    _check(_load().orc_sample_indices(seed, frame_id, M, l, _p(out)), "sample_indices")
    return out


def covariance(X: np.ndarray) -> np.ndarray:
    """X: complex64 (M, T) -> R complex128 (M, M)."""
    X = np.ascontiguousarray(X, dtype=np.complex64)
    M, T = X.shape
    R = np.zeros((M, M), dtype=np.complex128)
    _check(_load().orc_covariance(_p(X), M, T, T, _p(R)), "covariance")
    return R


def eigh_jacobi(A: np.ndarray, tol: float = 1e-14, max_sweeps: int = 60):
    A = _c128(A).copy()
    n = A.shape[0]
    w = np.zeros(n)
    V = np.zeros((n, n), dtype=np.complex128)
    sweeps = _check(_load().orc_eigh_jacobi(n, _p(A), _p(w), _p(V), tol, max_sweeps), "eigh_jacobi")
    return w, V, sweeps


def svd_jacobi(A: np.ndarray, tol: float = 1e-13, max_sweeps: int = 60):
    A = _c128(A)
    m, n = A.shape
    U = np.zeros((m, n), dtype=np.complex128)
    s = np.zeros(n)
    W = np.zeros((n, n), dtype=np.complex128)
    _check(_load().orc_svd_jacobi(m, n, _p(A), _p(U), _p(s), _p(W), tol, max_sweeps), "svd_jacobi")
    return U, s, W


def householder_qr(A: np.ndarray):
    A = _c128(A)
    m, n = A.shape
    Q = np.zeros((m, n), dtype=np.complex128)
    R = np.zeros((n, n), dtype=np.complex128)
    _check(_load().orc_householder_qr(m, n, _p(A), _p(Q), _p(R)), "householder_qr")
    return Q, R


def pinv_hermitian(H: np.ndarray):
    H = _c128(H)
    n = H.shape[0]
    W = np.zeros((n, n), dtype=np.complex128)
    rank = _check(_load().orc_pinv_hermitian(n, _p(H), _p(W)), "pinv_hermitian")
    return W, rank


def music_subspace(R: np.ndarray, K: int):
    R = _c128(R)
    M = R.shape[0]
    U = np.zeros((M, K), dtype=np.complex128)
    lam = np.zeros(M)
    _check(_load().orc_music_subspace(_p(R), M, K, _p(U), _p(lam)), "music_subspace")
    return U, lam


def fast_music(R: np.ndarray, K: int, l: int, t: int, method: int, seed: int, frame_id: int = 0,
               ncols: int | None = None, form: int = 0):
    """Randomized signal subspace (Algorithm 1 for method=1, Algorithm 2 for method=2).

    Returns (U, lamB, idx): U is M x ncols (ncols = K default, or l), lamB the l
    eigenvalues of B (descending), idx the sampled indices (method 1)."""
    R = _c128(R)
    M = R.shape[0]
    ncols = K if ncols is None else ncols
    U = np.zeros((M, ncols), dtype=np.complex128)
    lamB = np.zeros(l)
    idx = np.zeros(l, dtype=np.int32)
    _check(_load().orc_fast_music(_p(R), M, K, l, t, method, seed, frame_id, ncols, form,
                                  _p(U), _p(lamB), _p(idx)), "fast_music")
    return U, lamB, idx


def _positions(pos, M):
    """float64 copy of the element positions (wavelengths), or None for a uniform array."""
    if pos is None:
        return None
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    if pos.shape != (M,):
        raise ValueError(f"pos must hold M = {M} element positions")
    return pos


def spectrum(U: np.ndarray, theta0_deg: float, step_deg: float, L: int, d: float = 0.5,
             residual_form: bool = False, pos=None) -> np.ndarray:
    """Pseudo-spectrum on the grid; pos = element positions in wavelengths (None: d * m)."""
    U = _c128(U)
    M, nc = U.shape
    P = np.zeros(L)
    pp = _positions(pos, M)
    _check(_load().orc_spectrum(_p(U), M, nc, d, None if pp is None else _p(pp), theta0_deg, step_deg, L,
                                int(residual_form), _p(P)), "spectrum")
    return P


def peaks(P: np.ndarray, K: int):
    P = np.ascontiguousarray(P, dtype=np.float64)
    idx = np.zeros(K, dtype=np.int32)
    n = ctypes.c_int(0)
    _check(_load().orc_peaks(_p(P), P.shape[0], K, _p(idx), ctypes.byref(n)), "peaks")
    return idx, n.value


def frame(X: np.ndarray, K: int, l: int, t: int, method: int, seed: int, frame_id: int,
          theta0_deg: float, step_deg: float, L: int, d: float = 0.5, pos=None):
    """Whole frame: X (complex64 M x T) -> (P, peak_idx, n_peaks); pos = element positions
    in wavelengths (None: a uniform array of spacing d)."""
    X = np.ascontiguousarray(X, dtype=np.complex64)
    M, T = X.shape
    P = np.zeros(L)
    idx = np.zeros(K, dtype=np.int32)
    n = ctypes.c_int(0)
    pp = _positions(pos, M)
    _check(_load().orc_frame(_p(X), M, T, T, K, l, t, method, seed, frame_id, d,
                             None if pp is None else _p(pp), theta0_deg, step_deg, L, _p(P), _p(idx),
                             ctypes.byref(n)), "frame")
    return P, idx, n.value

"""Seeded synthetic radar frames (input generator shared by tests, smoke and bench).

This module holds only the data model of the paper's simulations -- the
far-field ULA received-signal model of Sec. II-A with half-wavelength spacing,
circular complex Gaussian sources and white complex Gaussian noise -- and the
workload shapes the benchmarks use.  It contains none of the estimator's
arithmetic (no covariance, sketch, subspace, spectrum or peak search), so both
the CUDA path and the FP64 oracle can be fed from it.  numpy only; it never
loads the CUDA library.

Signal model (Sec. II-A):  x_m(t) = sum_k a_m(theta_k) s_k(t) + n_m(t), with
a_m(theta) = exp(j 2 pi d m sin theta) (d in wavelengths, 0.5 = lambda/2) for a
uniform array, or exp(j 2 pi x_m sin theta) for element positions x_m,
s_k(t) ~ CN(0, P_k) i.i.d. over snapshots and n_m(t) ~ CN(0, sigma^2), i.e.
(N(0, sigma^2) + j N(0, sigma^2)) / sqrt(2).  SNR_k = 10 log10(P_k / sigma^2).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def rng_for(seed: int, stream: int = 0) -> np.random.Generator:
    """Philox-backed numpy generator; `stream` separates independent draws."""
    return np.random.Generator(np.random.Philox(key=[seed & 0xFFFFFFFFFFFFFFFF, stream]))


def draw_angles(rng: np.random.Generator, K: int, lo: float, hi: float, min_sep: float,
                max_tries: int = 100000) -> np.ndarray:
    """K angles (degrees) uniform in [lo, hi], sorted, pairwise gap >= min_sep
    (rejection sampling of the whole sorted set)."""
    for _ in range(max_tries):
        a = np.sort(rng.uniform(lo, hi, size=K))
        if K < 2 or np.min(np.diff(a)) >= min_sep:
            return a
    raise RuntimeError("could not place angles with the requested separation")


def ula_snapshots(rng: np.random.Generator, M: int, T: int, angles_deg, powers, sigma2: float,
                  d: float = 0.5) -> np.ndarray:
    """One frame X (M x T, complex64, row = antenna) of the Sec. II-A model."""
    angles = np.deg2rad(np.asarray(angles_deg, dtype=np.float64))
    powers = np.asarray(powers, dtype=np.float64)
    K = angles.shape[0]
    m = np.arange(M, dtype=np.float64)[:, None]
    A = np.exp(1j * 2.0 * np.pi * d * m * np.sin(angles)[None, :])  # M x K
    S = (rng.standard_normal((K, T)) + 1j * rng.standard_normal((K, T))) * np.sqrt(powers / 2.0)[:, None]
    N = (rng.standard_normal((M, T)) + 1j * rng.standard_normal((M, T))) * np.sqrt(sigma2 / 2.0)
    X = A @ S + N
    return X.astype(np.complex64)


def array_snapshots(rng: np.random.Generator, pos_wl, T: int, angles_deg, powers, sigma2: float) -> np.ndarray:
    """One frame X (M x T, complex64) of the Sec. II-A model for a linear array whose
    element m sits at pos_wl[m] wavelengths: a_m(theta) = exp(j 2 pi x_m sin theta)."""
    x = np.asarray(pos_wl, dtype=np.float64)[:, None]
    angles = np.deg2rad(np.asarray(angles_deg, dtype=np.float64))
    powers = np.asarray(powers, dtype=np.float64)
    K = angles.shape[0]
    M = x.shape[0]
    A = np.exp(1j * 2.0 * np.pi * x * np.sin(angles)[None, :])  # M x K
    S = (rng.standard_normal((K, T)) + 1j * rng.standard_normal((K, T))) * np.sqrt(powers / 2.0)[:, None]
    N = (rng.standard_normal((M, T)) + 1j * rng.standard_normal((M, T))) * np.sqrt(sigma2 / 2.0)
    return (A @ S + N).astype(np.complex64)


def sparse_virtual_array(M: int, seed: int = 0, fill: float = 0.75, jitter_wl: float = 0.02) -> np.ndarray:
    """Element positions (wavelengths, ascending) of a sparse virtual array: M of the
    ceil(M / fill) sites of a half-wavelength lattice, drawn at random (the first and
    last site always kept), each moved by a uniform offset in +-jitter_wl (residual
    placement error of a cascaded MIMO layout).  Non-uniform and off the lattice."""
    rng = rng_for(seed, 40000 + M)
    n_sites = int(np.ceil(M / fill))
    inner = rng.choice(np.arange(1, n_sites - 1), size=M - 2, replace=False)
    sites = np.sort(np.concatenate([[0, n_sites - 1], inner]))
    return 0.5 * sites + rng.uniform(-jitter_wl, jitter_wl, size=M)


@dataclass
class Frame:
    X: np.ndarray            # complex64, M x T
    angles_deg: np.ndarray   # true source angles
    snr_db: np.ndarray
    K: int
    l: int
    t: int
    theta0: float            # grid start (degrees)
    step: float              # grid step (degrees)
    L: int                   # grid points
    frame_id: int
    d: float = 0.5
    pos: np.ndarray | None = None   # element positions (wavelengths); None: uniform spacing d

    @property
    def M(self) -> int:
        return self.X.shape[0]

    @property
    def T(self) -> int:
        return self.X.shape[1]


@dataclass
class Workload:
    name: str
    frames: list = field(default_factory=list)


def _grid(lo: float, hi: float, step: float):
    L = int(round((hi - lo) / step)) + 1
    return lo, step, L


def small_frame(seed: int = 0) -> Frame:
    """ULA M=64, K=3 unit-power sources at -20, 5, 30 deg, T=200, SNR 10 dB,
    l = K + 10, t = 2, grid -90:0.1:90 (1801 points)."""
    rng = rng_for(seed, 1)
    ang = np.array([-20.0, 5.0, 30.0])
    sigma2 = 10.0 ** (-10.0 / 10.0)
    X = ula_snapshots(rng, 64, 200, ang, np.ones(3), sigma2)
    th0, st, L = _grid(-90.0, 90.0, 0.1)
    return Frame(X, ang, np.full(3, 10.0), 3, 13, 2, th0, st, L, frame_id=0)


def massive_mimo_frames(n_frames: int, seed: int = 0, M: int = 512, T: int = 1024, K: int = 8,
                        extra: int = 16, t: int = 1, fov: float = 60.0, min_sep: float = 2.0,
                        snr_lo: float = 0.0, snr_hi: float = 20.0, grid=(-75.0, 75.0, 0.01)) -> Workload:
    """Massive-MIMO frames: ULA M=512, K=8 sources uniform in +-60 deg with >= 2 deg
    gaps, T=1024, per-source SNR U(0, 20) dB, l = K + 16, one power iteration,
    grid -75:0.01:75 (15001 points).  Noise power 1."""
    wl = Workload(f"ula_M{M}_T{T}_K{K}_l{K + extra}_L{_grid(*grid)[2]}")
    th0, st, L = _grid(*grid)
    for b in range(n_frames):
        rng = rng_for(seed, 1000 + b)
        ang = draw_angles(rng, K, -fov, fov, min_sep)
        snr = rng.uniform(snr_lo, snr_hi, size=K)
        X = ula_snapshots(rng, M, T, ang, 10.0 ** (snr / 10.0), 1.0)
        wl.frames.append(Frame(X, ang, snr, K, K + extra, t, th0, st, L, frame_id=b))
    return wl


def precision_study_frames(n_frames: int, seed: int = 0) -> Workload:
    """ULA M=1024, K=16, +-60 deg with >= 1 deg gaps, T=2048, SNR U(5, 25) dB,
    l=48, t=1, grid -90:0.005:90 (36001 points)."""
    wl = massive_mimo_frames(n_frames, seed, M=1024, T=2048, K=16, extra=32, t=1, fov=60.0,
                             min_sep=1.0, snr_lo=5.0, snr_hi=25.0, grid=(-90.0, 90.0, 0.005))
    wl.name = "ula_M1024_T2048_K16_l48_L36001"
    return wl


def sparse_array_frames(n_frames: int, seed: int = 0, M: int = 256, T: int = 512, K: int = 6, extra: int = 10,
                        t: int = 1, fov: float = 50.0, snr_lo: float = 10.0, snr_hi: float = 20.0,
                        grid=(-60.0, 60.0, 0.02)) -> Workload:
    """Frames of one sparse virtual array (sparse_virtual_array(M, seed)): K sources in
    +-fov deg at least 3 beamwidths apart (beamwidth ~ 1 / aperture in sin(theta)),
    per-source SNR U(snr_lo, snr_hi) dB, noise power 1, l = K + extra."""
    pos = sparse_virtual_array(M, seed)
    aperture = pos.max() - pos.min()
    sep = 3.0 * np.rad2deg(1.0 / aperture)
    wl = Workload(f"sparse_M{M}_T{T}_K{K}_aperture{aperture:.1f}wl")
    th0, st, L = _grid(*grid)
    for b in range(n_frames):
        rng = rng_for(seed, 50000 + b)
        ang = draw_angles(rng, K, -fov, fov, sep)
        snr = rng.uniform(snr_lo, snr_hi, size=K)
        X = array_snapshots(rng, pos, T, ang, 10.0 ** (snr / 10.0), 1.0)
        wl.frames.append(Frame(X, ang, snr, K, K + extra, t, th0, st, L, frame_id=b, pos=pos))
    return wl


def uneven_frames(n_frames: int, seed: int = 0) -> Workload:
    """Uneven batch: M from {128,192,256,384,512}, T log-uniform in [64, 2048],
    K uniform in [1, 12], SNR U(0, 20) dB, l = K + 12, t = 1, grid -75:0.05:75."""
    wl = Workload("uneven_M128-512_T64-2048_K1-12")
    th0, st, L = _grid(-75.0, 75.0, 0.05)
    for b in range(n_frames):
        rng = rng_for(seed, 5000 + b)
        M = int(rng.choice([128, 192, 256, 384, 512]))
        T = int(round(np.exp(rng.uniform(np.log(64), np.log(2048)))))
        K = int(rng.integers(1, 13))
        ang = draw_angles(rng, K, -60.0, 60.0, 2.0)
        snr = rng.uniform(0.0, 20.0, size=K)
        X = ula_snapshots(rng, M, T, ang, 10.0 ** (snr / 10.0), 1.0)
        wl.frames.append(Frame(X, ang, snr, K, min(K + 12, M), 1, th0, st, L, frame_id=b))
    return wl


SERVING_PROFILES = {
    # name: (M, T, K_max, fov_deg, grid_step_deg)
    "long_range": (256, 256, 4, 9.0, 0.005),
    "medium_range": (384, 512, 8, 15.0, 0.01),
    "short_range": (512, 1024, 16, 75.0, 0.02),
}


def serving_frame(profile: str, frame_id: int, seed: int = 0) -> Frame:
    """One request of the serving mix: angles within 0.8 x FOV, gap >= 2 beamwidths
    (beamwidth ~ 2/M in sin(theta) -> degrees at broadside), K uniform in [1, K_max],
    SNR U(0, 20) dB, l = K + 12, t = 1."""
    M, T, kmax, fov, step = SERVING_PROFILES[profile]
    rng = rng_for(seed, 20000 + frame_id)
    K = int(rng.integers(1, kmax + 1))
    bw_deg = np.rad2deg(2.0 / M)
    ang = draw_angles(rng, K, -0.8 * fov, 0.8 * fov, 2.0 * bw_deg)
    snr = rng.uniform(0.0, 20.0, size=K)
    X = ula_snapshots(rng, M, T, ang, 10.0 ** (snr / 10.0), 1.0)
    th0, st, L = _grid(-fov, fov, step)
    return Frame(X, ang, snr, K, K + 12, 1, th0, st, L, frame_id=frame_id)


def bounds_study_frame(seed: int, M: int = 200, T: int = 400, K: int = 9, snr_db: float = 1.0,
                       lo: float = 0.0, hi: float = 80.0) -> Frame:
    """Frame of the error-bound experiment (Sec. V-C): K=9 sources in [0, 80] deg,
    M=200, N=2M, SNR 1 dB."""
    rng = rng_for(seed, 30000)
    ang = draw_angles(rng, K, lo, hi, 2.0)
    X = ula_snapshots(rng, M, T, ang, np.full(K, 10.0 ** (snr_db / 10.0)), 1.0)
    th0, st, L = _grid(-90.0, 90.0, 0.1)
    return Frame(X, ang, np.full(K, snr_db), K, K, 2, th0, st, L, frame_id=seed)

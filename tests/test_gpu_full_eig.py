"""Standard MUSIC (full eigendecomposition, Sec. II-B, Eq. 4-6) on the GPU, the comparison
method the benchmark times beside fast MUSIC, against the oracle's standard MUSIC
(hand-written FP64 Jacobi EVD) on the same complex64 frames.

Tolerances: the FP32 covariance and FP32 eigh move the signal subspace by eps =
||U U^H - U_o U_o^H||_F (measured, required <= 1e-4), so every denominator differs by at
most M eps plus the scan's rounding 8 u M K; peaks equal the oracle's for
well-separated sources at SNR >= 10 dB (the workloads below)."""
import numpy as np
import pytest

import oracle
from paper_1911_07434_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1911_07434_gb300 import binding, build
    build.build()
    c = binding.Context(device=0)
    yield c
    c.close()


def _cases():
    small = synth.small_frame()
    big = synth.massive_mimo_frames(1, seed=7, snr_lo=10.0, snr_hi=20.0).frames  # oracle EVD ~30 s
    return {"M64": [small], "M512": big}


@pytest.mark.parametrize("case", ["M64", "M512"])
def test_full_eig_music_matches_oracle(ctx, case):
    from paper_1911_07434_gb300.full_eig import full_eig_music
    frames = _cases()[case]
    f0 = frames[0]
    X = torch.from_numpy(np.stack([f.X for f in frames])).cuda()
    P, Uk, idx, deg, n = full_eig_music(ctx, X, f0.K, f0.theta0, f0.step, f0.L)
    torch.cuda.synchronize()
    for b, fr in enumerate(frames):
        # the oracle's standard-MUSIC frame (oracle.frame with FULL_EIG) step by step, so its
        # one Jacobi EVD serves both the subspace and the spectrum
        Uo, _ = oracle.music_subspace(oracle.covariance(fr.X), fr.K)
        Po = oracle.spectrum(Uo, fr.theta0, fr.step, fr.L)
        io, no = oracle.peaks(Po, fr.K)
        U = Uk[b].cpu().numpy().astype(np.complex128)
        eps = np.linalg.norm(U @ U.conj().T - Uo @ Uo.conj().T)
        assert eps <= 1e-4, eps
        Pg = P[b].cpu().numpy().astype(np.float64)
        M = fr.M
        assert np.max(np.abs(1.0 / Pg - 1.0 / Po)) <= M * eps + 8 * U32 * M * fr.K
        assert int(n[b]) == no == fr.K
        assert sorted(idx[b].cpu().tolist()) == sorted(io.tolist())
        est = np.sort(fr.theta0 + fr.step * io)
        assert np.max(np.abs(est - np.sort(fr.angles_deg))) < 0.3

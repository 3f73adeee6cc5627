"""Precision modes (FM_PREC_TF32 / FM_PREC_BF16) and the FP32 refinement step.

* Covariance: with operand unit roundoff u_p (TF32 2^-11, BF16 2^-8) every product
  carries a relative error below 2 u_p + u_p^2, so |R_ij - exact| <= (2.01 u_p +
  (T/4 + 16) u) S_ij with S_ij = sum_t |x_it| |x_jt| / T (u = 2^-24; the second term
  is the FP32 accumulator's, as in the 3xTF32 parity test).
* refine = 1 adds the power step V = orth(C), C = R V computed from X in FP32; in exact
  arithmetic that is the oracle run with t + 1 power steps, so FP32 + refine must meet
  the FP32 projector bound (1e-5) against oracle(t + 1), and so must TF32 and BF16 +
  refine: the step hands the final solve an FP32 image of R, which wins back what the
  low-precision covariance lost.
* Without refine, the projector error is a property of the precision, reported and
  bounded here by ten times what FP32 operands with the same arithmetic would give
  at u_p in place of u (measured: TF32 ~2.3e-4, BF16 ~1.9e-3 at M = 1024).
In every mode the peak indices equal the oracle's (sources >= 2 beamwidths apart,
SNR >= 10 dB here).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1911_07434_gb300 import synth  # noqa: E402

U32 = 2.0 ** -24
UP = {1: 2.0 ** -11, 2: 2.0 ** -8}


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1911_07434_gb300 import binding, build
    build.build()
    c = binding.Context(device=0)
    yield c
    c.close()


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("M,T", [(64, 200), (200, 1000), (256, 96)])
def test_covariance_precision_modes(ctx, prec, M, T):
    rng = np.random.default_rng(M + T + prec)
    X = ((rng.standard_normal((M, T)) + 1j * rng.standard_normal((M, T))) * rng.uniform(0.1, 10, (M, 1)))
    X = X.astype(np.complex64)
    R = ctx.covariance(torch.from_numpy(X).cuda(), prec=prec)[0].cpu().numpy().astype(np.complex128)
    Ro = oracle.covariance(X)
    A = np.abs(X.astype(np.complex128))
    S = A @ A.T / T
    bound = (2.01 * UP[prec] + (T / 4 + 16) * U32) * S
    assert np.all(np.abs(R - Ro) <= bound), np.max(np.abs(R - Ro) / S)
    # the error is of the operand precision's size, not far below it (the mode is really taken)
    assert np.max(np.abs(R - Ro) / S) > 0.05 * UP[prec]


def _frames(n, M=256, T=512, K=6, l=20, seed=21):
    return synth.massive_mimo_frames(n, seed=seed, M=M, T=T, K=K, extra=l - K, snr_lo=10.0, snr_hi=20.0,
                                     grid=(-70.0, 70.0, 0.05))


def _run(ctx, wl, method, prec, refine):
    fs, keep = [], []
    for fr in wl.frames:
        X = torch.from_numpy(np.ascontiguousarray(fr.X)).cuda()
        P = torch.empty(fr.L, dtype=torch.float32, device="cuda")
        idx = torch.empty(fr.K, dtype=torch.int32, device="cuda")
        deg = torch.empty(fr.K, dtype=torch.float32, device="cuda")
        n = torch.empty(1, dtype=torch.int32, device="cuda")
        st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        fs.append(ctx.frame(X, fr.K, fr.l, fr.t, method, fr.theta0, fr.step, fr.L, P, idx, deg, n, seed=5,
                            frame_id=fr.frame_id, status=st, prec=prec, refine=refine))
        keep.append((X, P, idx, st, deg, n))  # every buffer the frame points to stays alive
    ctx.run(fs)
    torch.cuda.synchronize()
    out = []
    for b, (fr, (X, P, idx, st, _, _)) in enumerate(zip(wl.frames, keep)):
        U = ctx.run_subspace(b, fr.X.shape[0], fr.K).cpu().numpy().astype(np.complex128)
        out.append((U, P.cpu().numpy().astype(np.float64), idx.cpu().numpy(), int(st.item())))
    return out


def _proj_err(U, Uo):
    return np.linalg.norm(U @ U.conj().T - Uo @ Uo.conj().T)


@pytest.mark.parametrize("method", [1, 2])
@pytest.mark.parametrize("prec,refine,bound", [(0, 1, 1e-5), (1, 1, 1e-5), (2, 1, 1e-5), (1, 0, 2.5e-3),
                                               (2, 0, 2e-2)])
def test_precision_modes_against_oracle(ctx, method, prec, refine, bound):
    wl = _frames(3)
    got = _run(ctx, wl, method, prec, refine)
    for fr, (U, P, idx, st) in zip(wl.frames, got):
        assert st == 0
        R = oracle.covariance(fr.X)
        Uo, _, _ = oracle.fast_music(R, fr.K, fr.l, fr.t + refine, method, 5, fr.frame_id)
        err = _proj_err(U, Uo)
        assert err <= bound, (prec, refine, err)
        Po = oracle.spectrum(Uo, fr.theta0, fr.step, fr.L)
        io, no = oracle.peaks(Po, fr.K)
        assert no == fr.K
        assert np.array_equal(np.sort(io), np.sort(idx))


def test_refine_rejected_without_snapshots(ctx):
    from paper_1911_07434_gb300 import binding
    R = torch.eye(32, dtype=torch.complex64, device="cuda")
    with pytest.raises(binding.FmError):
        ctx._check(binding.fm_subspace(ctx.h, R.data_ptr(), 1, 32, binding.FmParams(2, 2, 8, 1, 0, 0, 1, 0, 0), 0,
                                       torch.empty((32, 2), dtype=torch.complex64, device="cuda").data_ptr(),
                                       None, None), "fm_subspace")


def test_fp32_projector_at_precision_study_size(ctx):
    """The FP32 target (projector <= 1e-5 against the oracle) at the largest workload,
    M = 1024, T = 2048, K = 16, l = 48: the eigensolver's stopping test and the
    Rayleigh-Ritz correction must hold up at l = 48 too."""
    wl = synth.precision_study_frames(2, seed=0)
    got = _run(ctx, wl, 2, 0, 0)
    for fr, (U, P, idx, st) in zip(wl.frames, got):
        assert st == 0
        Uo, _, _ = oracle.fast_music(oracle.covariance(fr.X), fr.K, fr.l, fr.t, 2, 5, fr.frame_id)
        assert _proj_err(U, Uo) <= 1e-5

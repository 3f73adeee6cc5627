"""Edge cases of the whole path through the C ABI: invalid and empty inputs, the
largest sizes the library takes, and the degenerate cases of the method.

* Invalid requests return FM_ERR_INVALID_ARG and launch nothing.
* Largest sizes: M = 1024, l = 48, a 65,536-point grid; sampled spectrum points against
  the oracle (every 64th angle and the main lobes) and the peaks at the true angles.
* A Jacobi sweep cap of 1 makes an ordinary frame report FM_ERR_NO_CONVERGENCE; the
  next frame on the same context, with the cap restored, is clean.
* Random sampling with l = M keeps every column, so fast MUSIC is exact MUSIC (the
  oracle's full Jacobi eigendecomposition): projector <= 1e-5.
* Noise-free rank-K data make H = V^H R V singular in exact arithmetic, which takes the
  eigenvalue pseudo-inverse path of the core matrix; U_s must still span the steering
  vectors (projector against the oracle's exact subspace <= 1e-4).
* The smallest arrays (M = 2) and grids (L = 1, 2) and a single snapshot (T = 1).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1911_07434_gb300 import synth  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1911_07434_gb300 import binding, build
    build.build()
    return binding


@pytest.fixture(scope="module")
def ctx(lib):
    c = lib.Context(device=0)
    yield c
    c.close()


class One:
    """Device buffers and the fm_frame of one frame (kept alive together)."""

    def __init__(self, lib, X, K, l, t, method, theta0, step, L, seed=3, frame_id=0):
        self.X = torch.from_numpy(np.ascontiguousarray(X)).cuda()
        self.P = torch.full((L,), -1.0, dtype=torch.float32, device="cuda")
        self.idx = torch.full((K,), -7, dtype=torch.int32, device="cuda")
        self.deg = torch.empty(K, dtype=torch.float32, device="cuda")
        self.n = torch.zeros(1, dtype=torch.int32, device="cuda")
        self.st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        self.f = lib.Context.frame(self.X, K, l, t, method, theta0, step, L, self.P, self.idx, self.deg, self.n,
                                   seed=seed, frame_id=frame_id, status=self.st)


def proj(U):
    return U @ U.conj().T


def test_invalid_requests_launch_nothing(lib, ctx):
    fr = synth.small_frame()
    good = One(lib, fr.X, fr.K, fr.l, fr.t, 2, fr.theta0, fr.step, fr.L)
    l0 = lib.fm_launch_count(ctx.h)
    with pytest.raises(lib.FmError):
        ctx.run([])                                     # no frames
    bad = []
    for field, value in (("K", fr.l + 1), ("l", 49), ("t", 9), ("T", 0), ("ldx", fr.X.shape[1] - 1)):
        f = lib.FmFrame.from_buffer_copy(good.f)
        if field in ("K", "l", "t"):
            setattr(f.p, field, value)
        else:
            setattr(f, field, value)
        bad.append(f)
    f = lib.FmFrame.from_buffer_copy(good.f)
    f.grid.L = 0
    bad.append(f)
    f = lib.FmFrame.from_buffer_copy(good.f)
    f.grid.L = 65537
    bad.append(f)
    f = lib.FmFrame.from_buffer_copy(good.f)
    f.arr.M = 1
    bad.append(f)
    f = lib.FmFrame.from_buffer_copy(good.f)
    f.p.method = 0                                      # full-eig MUSIC is not an fm_run method
    bad.append(f)
    f = lib.FmFrame.from_buffer_copy(good.f)
    f.P_out = None
    bad.append(f)
    for f in bad:
        with pytest.raises(lib.FmError):
            ctx.run([good.f, f])                        # one bad frame rejects the whole call
    assert lib.fm_launch_count(ctx.h) == l0
    ctx.run([good.f])
    torch.cuda.synchronize()
    assert int(good.st.item()) == 0


def test_largest_sizes(lib, ctx):
    """M = 1024, l = 48, K = 16 and the largest grid, L = 65,536 points (0.00275 deg)."""
    wl = synth.precision_study_frames(1, seed=3)
    fr = wl.frames[0]
    L = 65536
    step = 180.0 / (L - 1)
    one = One(lib, fr.X, fr.K, fr.l, fr.t, 2, -90.0, step, L, frame_id=fr.frame_id)
    ctx.run([one.f])
    torch.cuda.synchronize()
    assert int(one.st.item()) == 0 and int(one.n.item()) == fr.K
    Uo, _, _ = oracle.fast_music(oracle.covariance(fr.X), fr.K, fr.l, fr.t, 2, 3, fr.frame_id)
    U = ctx.run_subspace(0, 1024, fr.K).cpu().numpy().astype(np.complex128)
    eps = np.linalg.norm(proj(U) - proj(Uo))
    assert eps <= 1e-5
    # every 64th angle plus the 64 angles around each true source (main lobes included)
    th_all = -90.0 + step * np.arange(L)
    sel = np.arange(0, L, 64)
    for a in fr.angles_deg:
        c = int(round((a + 90.0) / step))
        sel = np.union1d(sel, np.arange(max(0, c - 32), min(L, c + 32)))
    Pg = one.P.cpu().numpy().astype(np.float64)[sel]
    Po = np.array([oracle.spectrum(Uo, th_all[i], step, 1)[0] for i in sel])
    th = th_all[sel]
    far = np.min(np.abs(th[:, None] - fr.angles_deg[None, :]), axis=1) > 2 * np.rad2deg(2.0 / 1024)
    assert np.max(np.abs(10 * np.log10(Pg[far] / Po[far]))) < 0.01
    # every sampled denominator: |a^H (U U^H - Uo Uo^H) a| <= M eps, plus the scan's rounding
    assert np.max(np.abs(1.0 / Pg - 1.0 / Po)) <= 1024 * eps + 16 * 2.0 ** -24 * 1024 * fr.K
    est = np.sort(one.deg.cpu().numpy())
    assert np.max(np.abs(est - np.sort(fr.angles_deg))) < 0.01


def test_sampling_all_columns_is_exact_music(lib, ctx):
    """Alg. 1 with l = M keeps every column: the sketch is R itself and U_s is the top-K
    eigenspace of R (exact MUSIC, Eq. 4)."""
    rng = synth.rng_for(5, 1)
    M, K = 40, 3
    X = synth.ula_snapshots(rng, M, 120, [-30.0, 0.0, 40.0], np.full(K, 10.0), 1.0)
    one = One(lib, X, K, M, 0, 1, -90.0, 0.5, 361)
    ctx.run([one.f])
    torch.cuda.synchronize()
    assert int(one.st.item()) == 0
    U = ctx.run_subspace(0, M, K).cpu().numpy().astype(np.complex128)
    Ue, _ = oracle.music_subspace(oracle.covariance(X), K)
    assert np.linalg.norm(proj(U) - proj(Ue)) <= 1e-5


@pytest.mark.parametrize("method", [1, 2])
def test_noise_free_rank_k_takes_the_pseudo_inverse_path(lib, ctx, method):
    """sigma = 0: R = A S S^H A^H / T has rank K < l, so H is singular and W is the
    eigenvalue pseudo-inverse; U_s still spans the steering vectors."""
    rng = synth.rng_for(6, 2)
    M, K, l = 64, 3, 10
    ang = [-25.0, 10.0, 35.0]
    X = synth.ula_snapshots(rng, M, 200, ang, np.ones(K), 0.0)
    one = One(lib, X, K, l, 1, method, -90.0, 0.1, 1801)
    ctx.run([one.f])
    torch.cuda.synchronize()
    U = ctx.run_subspace(0, M, K).cpu().numpy().astype(np.complex128)
    A = np.exp(1j * np.pi * np.arange(M)[:, None] * np.sin(np.deg2rad(ang))[None, :])
    Qa, _ = np.linalg.qr(A)
    assert np.linalg.norm(proj(U) - proj(Qa)) <= 1e-4
    est = np.sort(one.deg.cpu().numpy())
    assert np.max(np.abs(est - np.sort(ang))) <= 0.1


def test_smallest_array_grid_and_snapshot_count(lib, ctx):
    rng = synth.rng_for(7, 3)
    # M = 2, K = 1, l = 2, one snapshot
    X = synth.ula_snapshots(rng, 2, 1, [20.0], np.ones(1), 0.01)
    a = One(lib, X, 1, 2, 1, 2, -90.0, 1.0, 181)
    # a one-point grid and a two-point grid
    X2 = synth.ula_snapshots(rng, 16, 32, [0.0], np.ones(1), 0.1)
    b = One(lib, X2, 1, 4, 1, 2, 0.0, 1.0, 1)
    c = One(lib, X2, 1, 4, 1, 2, -1.0, 1.0, 2, frame_id=1)
    ctx.run([a.f, b.f, c.f])
    torch.cuda.synchronize()
    for o in (a, b, c):
        assert int(o.st.item()) == 0
    # M = 2: the spectrum against the oracle on the same data
    Uo, _, _ = oracle.fast_music(oracle.covariance(X), 1, 2, 1, 2, 3, 0)
    Po = oracle.spectrum(Uo, -90.0, 1.0, 181)
    Pg = a.P.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(1 / Pg - 1 / Po)) <= 1e-5 * 2
    # L = 1: the single point is a maximum; L = 2: the larger endpoint
    assert int(b.n.item()) == 1 and int(b.idx[0].item()) == 0
    Pc = c.P.cpu().numpy()
    assert int(c.n.item()) == 1 and int(c.idx[0].item()) == int(np.argmax(Pc))


def test_bounded_wait_reports_timeout_and_context_stays_usable(lib, ctx):
    """Failure detection without a GPU fault: a wait on a barrier nothing arrives on gives
    up after its limit, the status word carries FM_ERR_TIMEOUT, and the next frame runs."""
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    ctx._check(lib.fm_selftest_wait_timeout(ctx.h, st.data_ptr(), 2.0, None), "fm_selftest_wait_timeout")
    torch.cuda.synchronize()
    assert int(st.item()) == 1 << lib.FM_ERR_TIMEOUT
    fr = synth.small_frame()
    one = One(lib, fr.X, fr.K, fr.l, fr.t, 2, fr.theta0, fr.step, fr.L)
    ctx.run([one.f])
    torch.cuda.synchronize()
    assert int(one.st.item()) == 0 and int(one.n.item()) == fr.K


def test_sweep_cap_reports_no_convergence_and_next_frame_is_clean(lib, ctx):
    """Failure detection of the l x l eigensolves (Alg. 1 / 2's SVD / EVD steps, run as
    Jacobi sweeps): with one sweep allowed, the solve of an ordinary frame (l = 13)
    cannot converge, so its status word carries FM_ERR_NO_CONVERGENCE while every output
    stays finite; with the cap restored the next frame is clean and matches the oracle's
    peaks."""
    fr = synth.small_frame()
    one = One(lib, fr.X, fr.K, fr.l, fr.t, 2, fr.theta0, fr.step, fr.L)
    ctx.set_sweep_cap(1)
    try:
        ctx.run([one.f])
        torch.cuda.synchronize()
    finally:
        ctx.set_sweep_cap(0)
    assert int(one.st.item()) & (1 << lib.FM_ERR_NO_CONVERGENCE)
    assert not torch.isnan(one.P).any()
    two = One(lib, fr.X, fr.K, fr.l, fr.t, 2, fr.theta0, fr.step, fr.L)
    ctx.run([two.f])
    torch.cuda.synchronize()
    assert int(two.st.item()) == 0
    _, io, no = oracle.frame(fr.X, fr.K, fr.l, fr.t, 2, 3, 0, fr.theta0, fr.step, fr.L)
    assert int(two.n.item()) == no
    assert sorted(two.idx.cpu().tolist()) == sorted(io.tolist())
    with pytest.raises(lib.FmError):
        ctx.set_sweep_cap(31)

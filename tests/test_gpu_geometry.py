"""Non-uniform arrays (element positions fm_array.pos_wl, Sec. II-A signal model) through
the C ABI against the FP64 oracle with the same positions.

* fm_spectrum_array on random orthonormal U: every denominator within the uniform-array
  scan bound 8 u M ncols plus the extra steering rounding of the position split,
  0.01 |x|_max u M ncols (x_lo = x - x_hi is below 2^-11 |x|, |q| <= 2, one FP32 rounding
  of pi x_lo q per element, summed with |u_mk| over the rows: 2 ncols sqrt(M) sqrt(M)
  times that).
* fm_run on sparse virtual-array frames (both scan paths): the whole grid, main lobes
  included, with the bound of the end-to-end parity tests; peaks equal the oracle's.
* One fm_run mixing a uniform and a sparse array of the same M: each frame equals its run
  alone (peaks bit for bit, spectra within the scan tolerance).
"""
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


def proj(U):
    return U @ U.conj().T


@pytest.mark.parametrize("M,nc,grid", [(37, 3, (-89.0, 0.7, 255)), (96, 8, (-60.0, 0.02, 6001)),
                                       (256, 13, (-75.0, 0.05, 3001)), (1000, 16, (-90.0, 0.9, 201))])
def test_spectrum_array_parity(ctx, M, nc, grid):
    rng = np.random.default_rng(3 * M + nc)
    U = np.linalg.qr(rng.standard_normal((M, nc)) + 1j * rng.standard_normal((M, nc)))[0].astype(np.complex64)
    pos = synth.sparse_virtual_array(M, seed=M)
    th0, st, L = grid
    P = ctx.spectrum_array(torch.from_numpy(U).cuda(), th0, st, L, pos_wl=pos)[0].cpu().numpy().astype(np.float64)
    Po = oracle.spectrum(U.astype(np.complex128), th0, st, L, pos=pos)
    bound = (8 + 0.01 * np.max(np.abs(pos))) * U32 * M * nc
    assert np.max(np.abs(1.0 / P - 1.0 / Po)) <= bound, (np.max(np.abs(1.0 / P - 1.0 / Po)), bound)
    # uniform positions d m through the position path equal the uniform-array scan
    Pu = ctx.spectrum_array(torch.from_numpy(U).cuda(), th0, st, L, pos_wl=0.5 * np.arange(M))[0].cpu().numpy()
    Pd = ctx.spectrum(torch.from_numpy(U).cuda(), th0, st, L)[0].cpu().numpy()
    assert np.max(np.abs(1.0 / Pu.astype(np.float64) - 1.0 / Pd.astype(np.float64))) <= 8 * U32 * M * nc


def _frame_bufs(ctx, fr, method=2):
    X = torch.from_numpy(np.ascontiguousarray(fr.X)).cuda()
    P = torch.empty(fr.L, dtype=torch.float32, device="cuda")
    idx = torch.empty(fr.K, dtype=torch.int32, device="cuda")
    deg = torch.empty(fr.K, dtype=torch.float32, device="cuda")
    n = torch.empty(1, dtype=torch.int32, device="cuda")
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    f = ctx.frame(X, fr.K, fr.l, fr.t, method, fr.theta0, fr.step, fr.L, P, idx, deg, n, seed=3,
                  frame_id=fr.frame_id, status=st, pos_wl=fr.pos)
    return f, (X, P, idx, deg, n, st)


@pytest.mark.parametrize("path", ["tc", "simt"])
def test_run_sparse_array_every_angle(ctx, path):
    """Six frames of a sparse virtual array (M = 256, K = 6, aperture ~170 wavelengths)
    through fm_run, tensor-core or CUDA-core scan forced."""
    from paper_1911_07434_gb300 import binding
    wl = synth.sparse_array_frames(6, seed=1, M=256, T=512, K=6)
    ctx.set_scan_path(binding.FM_COV_TC if path == "tc" else binding.FM_COV_SIMT)
    try:
        bufs = [_frame_bufs(ctx, fr) for fr in wl.frames]
        ctx.run([b[0] for b in bufs])
        torch.cuda.synchronize()
        assert ctx.last_scan_path() == (binding.FM_COV_TC if path == "tc" else binding.FM_COV_SIMT)
        Us = [ctx.run_subspace(b, 256, 6).cpu().numpy().astype(np.complex128) for b in range(len(bufs))]
    finally:
        ctx.set_scan_path(binding.FM_COV_AUTO)
    xmax = np.max(np.abs(wl.frames[0].pos))
    for b in (0, 3):
        fr = wl.frames[b]
        X, P, idx, deg, n, st = bufs[b][1]
        assert int(st[0]) == 0
        R = oracle.covariance(fr.X)
        Uo, _, _ = oracle.fast_music(R, fr.K, fr.l, fr.t, 2, 3, fr.frame_id)
        Po = oracle.spectrum(Uo, fr.theta0, fr.step, fr.L, pos=fr.pos)
        io, no = oracle.peaks(Po, fr.K)
        eps = np.linalg.norm(proj(Us[b]) - proj(Uo))
        assert eps <= 1e-5, eps
        Pg = P.cpu().numpy().astype(np.float64)
        bound = fr.M * eps + ((16 if path == "tc" else 8) + 0.01 * xmax) * U32 * fr.M * fr.K
        assert np.max(np.abs(1.0 / Pg - 1.0 / Po)) <= bound
        assert int(n[0]) == no == fr.K
        assert sorted(idx.cpu().tolist()) == sorted(io.tolist())
        assert np.max(np.abs(Pg[io] / Po[io] - 1.0)) <= 1e-2
        est = np.sort(deg.cpu().numpy())
        assert np.max(np.abs(est - np.sort(fr.angles_deg))) < 0.1


def test_mixed_geometries_in_one_run(ctx):
    """A uniform and a sparse array of the same M in one fm_run: the scan keeps their
    steering apart (separate scan groups), and each frame equals its run alone."""
    sparse = synth.sparse_array_frames(4, seed=4, M=128, T=256, K=3, extra=9).frames
    ula = synth.massive_mimo_frames(4, seed=4, M=128, T=256, K=3, extra=9, grid=(-60.0, 60.0, 0.02)).frames
    for i, fr in enumerate(ula):
        fr.frame_id = 100 + i
    mixed = [sparse[0], ula[0], sparse[1], ula[1], sparse[2], ula[2], sparse[3], ula[3]]
    bufs = [_frame_bufs(ctx, fr) for fr in mixed]
    ctx.run([b[0] for b in bufs])
    torch.cuda.synchronize()
    for fr, (f, out) in zip(mixed, bufs):
        alone = _frame_bufs(ctx, fr)
        ctx.run([alone[0]])
        torch.cuda.synchronize()
        assert int(out[5][0]) == 0 and int(alone[1][5][0]) == 0
        assert torch.equal(out[2], alone[1][2])
        a = out[1].cpu().numpy().astype(np.float64)
        b = alone[1][1].cpu().numpy().astype(np.float64)
        xmax = 0.5 * fr.M if fr.pos is None else np.max(np.abs(fr.pos))
        assert np.max(np.abs(1.0 / a - 1.0 / b)) <= (16 + 0.01 * xmax) * U32 * fr.M * fr.K

"""The tensor-core sketch (Alg. 1 / Alg. 2 products C = R Omega and the power steps
C = R V of Eq. 11) through fm_run, against the FP64 oracle and against the CUDA-core
sketch on the same frames.

In FP32 mode the last product of a frame takes three TF32 MMAs per FP32 product
(hi*hi + hi*lo + lo*hi, relative error below 3 * 2^-22 per product) and the products
before it one TF32 MMA; the final solve reads only the last product, so U_s keeps the
1e-5 projector bound of the FP32 path.  The cases cover a single partial row tile
(M < 128), a ragged second tile, a partial last K chunk (2M not a multiple of 16), the
largest sketch (l = 48: 96 B rows), t = 0 (the first product is the last), sampling
with a power step, and frames of different shapes in one call.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1911_07434_gb300 import synth  # noqa: E402

# (M, T, K, l, t, method)
CASES = [
    (64, 200, 3, 13, 0, 2),
    (100, 150, 5, 7, 1, 2),
    (130, 333, 4, 16, 2, 2),
    (200, 400, 6, 24, 1, 1),
    (258, 300, 8, 48, 1, 2),
    (512, 1024, 8, 24, 1, 2),
    (6, 10, 1, 2, 1, 2),
    (64, 128, 2, 5, 3, 1),
]


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


def proj(U):
    return U @ U.conj().T


class One:
    """Device buffers and the fm_frame of one frame (kept alive together)."""

    def __init__(self, lib, X, K, l, t, method, frame_id, prec=0, L=721):
        self.X = torch.from_numpy(np.ascontiguousarray(X)).cuda()
        self.P = torch.empty(L, dtype=torch.float32, device="cuda")
        self.idx = torch.empty(K, dtype=torch.int32, device="cuda")
        self.deg = torch.empty(K, dtype=torch.float32, device="cuda")
        self.n = torch.zeros(1, dtype=torch.int32, device="cuda")
        self.st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        self.f = lib.Context.frame(self.X, K, l, t, method, -90.0, 0.25, L, self.P, self.idx, self.deg, self.n,
                                   seed=9, frame_id=frame_id, status=self.st, prec=prec)


def _frames(seed=0, cases=CASES):
    out = []
    for i, (M, T, K, l, t, method) in enumerate(cases):
        rng = synth.rng_for(seed + i, 31)
        ang = synth.draw_angles(rng, K, -60.0, 60.0, 2.5 * np.rad2deg(2.0 / M))
        X = synth.ula_snapshots(rng, M, T, ang, np.full(K, 10.0), 1.0)
        out.append((X, K, l, t, method, i))
    return out


def _run(lib, ctx, frames, path, prec=0):
    ctx.set_sketch_path(path)
    try:
        ones = [One(lib, X, K, l, t, m, fid, prec=prec) for X, K, l, t, m, fid in frames]
        ctx.run([o.f for o in ones])
        torch.cuda.synchronize()
        used = ctx.last_sketch_path()
        Us = [ctx.run_subspace(k, fr[0].shape[0], fr[1]).cpu().numpy().astype(np.complex128)
              for k, fr in enumerate(frames)]
    finally:
        ctx.set_sketch_path(lib.FM_COV_AUTO)
    for o in ones:
        assert int(o.st.item()) == 0
    return Us, used, ones


def test_tensor_core_sketch_against_oracle_and_cuda_cores(lib, ctx):
    frames = _frames()
    Ut, used_t, _ = _run(lib, ctx, frames, lib.FM_COV_TC)
    Us, used_s, _ = _run(lib, ctx, frames, lib.FM_COV_SIMT)
    assert used_t == lib.FM_COV_TC and used_s == lib.FM_COV_SIMT
    for (X, K, l, t, m, fid), ut, us in zip(frames, Ut, Us):
        Uo, _, _ = oracle.fast_music(oracle.covariance(X), K, l, t, m, 9, fid)
        et = np.linalg.norm(proj(ut) - proj(Uo))
        es = np.linalg.norm(proj(us) - proj(Uo))
        assert et <= 1e-5 and es <= 1e-5, (X.shape, l, t, m, et, es)
        assert np.linalg.norm(proj(ut) - proj(us)) <= 1e-5


def test_odd_m_falls_back_and_forced_path_refuses(lib, ctx):
    """R's rows are 8M bytes apart: an odd M cannot be read by TMA, so AUTO takes the
    CUDA-core sketch for that frame, and FM_COV_TC refuses the call before any launch."""
    frames = _frames(seed=50, cases=[(63, 100, 2, 6, 1, 2), (64, 100, 2, 6, 1, 2)])
    Ua, used, _ = _run(lib, ctx, frames, lib.FM_COV_AUTO)
    assert used == lib.FM_COV_AUTO  # one frame on each path
    for (X, K, l, t, m, fid), u in zip(frames, Ua):
        Uo, _, _ = oracle.fast_music(oracle.covariance(X), K, l, t, m, 9, fid)
        assert np.linalg.norm(proj(u) - proj(Uo)) <= 1e-5
    ctx.set_sketch_path(lib.FM_COV_TC)
    try:
        ones = [One(lib, X, K, l, t, m, fid) for X, K, l, t, m, fid in frames]
        l0 = lib.fm_launch_count(ctx.h)
        with pytest.raises(lib.FmError):
            ctx.run([o.f for o in ones])
        assert lib.fm_launch_count(ctx.h) == l0
    finally:
        ctx.set_sketch_path(lib.FM_COV_AUTO)


@pytest.mark.parametrize("prec", [1, 2])
def test_reduced_precision_frames_keep_one_mma_per_product(lib, ctx, prec):
    """TF32 / BF16 frames take every product with one TF32 MMA: the projector error is at
    the TF32 level (covariance and sketch operands rounded to a 10-bit mantissa, or BF16's 7
    bits in the covariance), well above FP32's but far below a wrong subspace."""
    frames = _frames(seed=70, cases=[(128, 256, 4, 12, 1, 2), (96, 200, 3, 8, 2, 1)])
    Ut, used, _ = _run(lib, ctx, frames, lib.FM_COV_TC, prec=prec)
    assert used == lib.FM_COV_TC
    for (X, K, l, t, m, fid), u in zip(frames, Ut):
        Uo, _, _ = oracle.fast_music(oracle.covariance(X), K, l, t, m, 9, fid)
        assert np.linalg.norm(proj(u) - proj(Uo)) <= 2e-2

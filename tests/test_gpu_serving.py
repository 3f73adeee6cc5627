"""Continuous-batching server (fm_serve_submit / fm_serve_poll) on the serving mix.

Each frame's result must be the same when it runs alone through fm_run and when it
is served inside a mix of frames of the three range profiles (M = 256 / 384 / 512,
different T, K, l and grids), within the scan tolerance: the tensor-core scan runs
per group of frames sharing M, U_s columns and grid, and a group's batch changes
with the mix, so the denominators M - ||U_s^H a||^2 may differ by rounding (bound
16 u M ncols, the tensor-core vs CUDA-core scan bound), and a peak may move by one
grid point only where the two neighbours' denominators are that close.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1911_07434_gb300 import synth  # noqa: E402

U32 = 2.0 ** -24
PROFILES = list(synth.SERVING_PROFILES)


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1911_07434_gb300 import binding, build
    build.build()
    return binding


class Req:
    def __init__(self, binding, fr):
        self.fr = fr
        self.X = torch.from_numpy(np.ascontiguousarray(fr.X)).cuda()
        self.P = torch.full((fr.L,), -1.0, dtype=torch.float32, device="cuda")
        self.idx = torch.full((fr.K,), -7, dtype=torch.int32, device="cuda")
        self.deg = torch.empty(fr.K, dtype=torch.float32, device="cuda")
        self.n = torch.zeros(1, dtype=torch.int32, device="cuda")
        self.st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        self.f = binding.Context.frame(self.X, fr.K, fr.l, fr.t, 2, fr.theta0, fr.step, fr.L, self.P, self.idx,
                                       self.deg, self.n, seed=11, frame_id=fr.frame_id, status=self.st)

    def result(self):
        return (self.P.cpu().numpy().astype(np.float64), self.idx.cpu().numpy().copy(), int(self.n.item()),
                int(self.st.item()))


def mix(binding, n, seed=3):
    return [Req(binding, synth.serving_frame(PROFILES[i % 3], frame_id=i, seed=seed)) for i in range(n)]


def serve_all(ctx, reqs, max_polls=2_000_000):
    tickets = [ctx.serve_submit(r.f) for r in reqs]
    pending = list(tickets)
    polls = 0
    while pending:
        pending = [t for t in pending if not ctx.serve_poll(t)]
        polls += 1
        assert polls < max_polls, "server did not finish"
    torch.cuda.synchronize()


def check_same(alone, mixed, fr):
    Pa, ia, na, sa = alone
    Pm, im, nm, sm = mixed
    assert sa == 0 and sm == 0 and na == nm == fr.K
    nc = fr.K  # rank-restricted U_s has K columns
    M = fr.X.shape[0]
    tol = 16 * U32 * M * nc
    da, dm = 1.0 / Pa, 1.0 / Pm
    j = int(np.argmax(np.abs(da - dm)))
    assert np.max(np.abs(da - dm)) <= tol, (np.max(np.abs(da - dm)), "M", M, "K", fr.K, "l", fr.l, "angle", j,
                                            da[j], dm[j], "first", da[0], dm[0], "peaks", sorted(ia), sorted(im))
    for a, b in zip(sorted(ia), sorted(im)):
        if a != b:  # only a near-tie of adjacent grid points may move a peak
            assert abs(int(a) - int(b)) == 1 and abs(da[a] - da[b]) <= 2 * tol


def test_served_mix_matches_each_frame_alone(lib):
    ctx = lib.Context(device=0)
    try:
        reqs = mix(lib, 48)
        serve_all(ctx, reqs)
        mixed = [r.result() for r in reqs]
        for r, m in zip(reqs, mixed):
            r.P.fill_(-1.0)
            r.idx.fill_(-7)
            ctx.run([r.f])
            torch.cuda.synchronize()
            check_same(r.result(), m, r.fr)
    finally:
        ctx.close()


def test_queued_frames_are_batched(lib):
    """Frames submitted faster than the slots drain are admitted as batches: far fewer
    kernel launches than one fm_run per frame, and every result complete."""
    ctx = lib.Context(device=0)
    try:
        one = mix(lib, 1, seed=5)
        ctx.run([one[0].f])
        torch.cuda.synchronize()
        per_frame = lib.fm_launch_count(ctx.h)
        reqs = mix(lib, 96, seed=5)
        base = lib.fm_launch_count(ctx.h)
        serve_all(ctx, reqs)
        used = lib.fm_launch_count(ctx.h) - base
        assert used < 0.6 * 96 * per_frame, (used, per_frame)
        for r in reqs:
            P, idx, n, st = r.result()
            assert st == 0 and n == r.fr.K and np.all(P > 0)
    finally:
        ctx.close()


def test_budget_admission(lib):
    """A budget with room for about one frame's workspace serves the mix one batch at a
    time with the same results; a frame larger than the budget is refused at submit."""
    reqs = mix(lib, 6, seed=9)
    need, largest = max((lib.fm_workspace_bytes([r.f]), i) for i, r in enumerate(reqs))
    big = lib.Context(device=0)
    small = lib.Context(budget_bytes=int(need * 1.3), device=0)
    try:
        serve_all(big, reqs)
        ref = [r.result() for r in reqs]
        for r in reqs:
            r.P.fill_(-1.0)
        serve_all(small, reqs)
        for r, a in zip(reqs, ref):
            check_same(a, r.result(), r.fr)
        tiny = lib.Context(budget_bytes=int(need // 4), device=0)
        try:
            with pytest.raises(lib.FmError):
                tiny.serve_submit(reqs[largest].f)
        finally:
            tiny.close()
    finally:
        small.close()
        big.close()

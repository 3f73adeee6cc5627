"""Independent contexts on separate streams run at the same time on one GPU (what the
serving slots do).  Every kernel of the path must give the same bits whatever runs beside
it: the same batch launched on four contexts at once, on four streams, must reproduce a
sequential run exactly (a missing barrier inside a kernel shows up here first, because
co-resident work changes the timing of its warps).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1911_07434_gb300 import synth  # noqa: E402

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
        self.P = torch.empty(fr.L, dtype=torch.float32, device="cuda")
        self.idx = torch.empty(fr.K, dtype=torch.int32, device="cuda")
        self.deg = torch.empty(fr.K, dtype=torch.float32, device="cuda")
        self.n = torch.zeros(1, dtype=torch.int32, device="cuda")
        self.st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        self.f = binding.Context.frame(self.X, fr.K, fr.l, fr.t, 2, fr.theta0, fr.step, fr.L, self.P, self.idx,
                                       self.deg, self.n, seed=11, frame_id=fr.frame_id, status=self.st)


def test_concurrent_contexts_reproduce_a_sequential_run(lib):
    frames = [synth.serving_frame(PROFILES[i % 3], frame_id=i, seed=5) for i in range(24)]
    copies = [[Req(lib, fr) for fr in frames] for _ in range(5)]  # [0]: sequential reference
    ctxs = [lib.Context(device=0) for _ in range(5)]
    streams = [torch.cuda.Stream() for _ in range(4)]
    rng = np.random.default_rng(7)
    try:
        for it in range(10):
            ids = list(rng.choice(len(frames), size=int(rng.integers(6, 16)), replace=False))
            ctxs[0].run([copies[0][k].f for k in ids])
            torch.cuda.synchronize()
            ref = {k: copies[0][k].P.cpu().numpy().copy() for k in ids}
            for j in range(4):
                for k in ids:
                    copies[j + 1][k].P.fill_(-1.0)
            torch.cuda.synchronize()
            for j in range(4):
                ctxs[j + 1].run([copies[j + 1][k].f for k in ids], stream=streams[j])
            torch.cuda.synchronize()
            for j in range(4):
                for k in ids:
                    r = copies[j + 1][k]
                    assert int(r.st.item()) == 0
                    assert np.array_equal(r.P.cpu().numpy(), ref[k]), (it, j, k, r.fr.X.shape)
    finally:
        for c in ctxs:
            c.close()

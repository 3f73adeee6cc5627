"""Uneven batches: grouped tensor-core scan, CUDA-graph replay and the path autotuner.

* The uneven workload (M in {128 ... 512}, T log-uniform in [64, 2048], K in [1, 12],
  l = K + 12) splits into many scan groups; its tensor-core path must agree with the
  CUDA-core path within the scan tolerance (16 u M ncols on every denominator) and
  pick the same peaks.
* A CUDA graph of the chain replays exactly the kernels fm_run launches, so its
  outputs equal fm_run's bit for bit, also after the inputs change between launches.
* fm_autotune leaves the context on a path combination that runs the frames.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1911_07434_gb300 import synth  # noqa: E402

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1911_07434_gb300 import binding, build
    build.build()
    return binding


class Batch:
    def __init__(self, binding, wl):
        self.wl = wl
        self.bufs, self.frames = [], []
        for fr in wl.frames:
            X = torch.from_numpy(np.ascontiguousarray(fr.X)).cuda()
            P = torch.full((fr.L,), -1.0, dtype=torch.float32, device="cuda")
            idx = torch.full((fr.K,), -7, dtype=torch.int32, device="cuda")
            deg = torch.empty(fr.K, dtype=torch.float32, device="cuda")
            n = torch.zeros(1, dtype=torch.int32, device="cuda")
            st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
            self.bufs.append((X, P, idx, deg, n, st))
            self.frames.append(binding.Context.frame(X, fr.K, fr.l, fr.t, 2, fr.theta0, fr.step, fr.L, P, idx, deg,
                                                     n, seed=3, frame_id=fr.frame_id, status=st))

    def results(self):
        torch.cuda.synchronize()
        return [(P.cpu().numpy().copy(), idx.cpu().numpy().copy(), int(st.item())) for X, P, idx, deg, n, st in self.bufs]

    def clear(self):
        for X, P, idx, deg, n, st in self.bufs:
            P.fill_(-1.0)
            idx.fill_(-7)


def test_uneven_batch_tensor_core_scan_groups(lib):
    ctx = lib.Context(device=0)
    try:
        b = Batch(lib, synth.uneven_frames(40, seed=4))
        out = {}
        for path in (lib.FM_COV_SIMT, lib.FM_COV_TC):
            ctx.set_scan_path(path)
            b.clear()
            ctx.run(b.frames)
            assert ctx.last_scan_path() == path
            out[path] = b.results()
        for fr, (Ps, is_, ss), (Pt, it, stt) in zip(b.wl.frames, out[lib.FM_COV_SIMT], out[lib.FM_COV_TC]):
            assert ss == 0 and stt == 0
            M = fr.X.shape[0]
            tol = 16 * U32 * M * fr.K
            d = np.abs(1.0 / Ps.astype(np.float64) - 1.0 / Pt.astype(np.float64))
            assert d.max() <= tol, (M, fr.K, d.max())
            for a, c in zip(np.sort(is_), np.sort(it)):
                assert a == c or (abs(int(a) - int(c)) == 1 and abs(1 / Ps[a] - 1 / Ps[c]) <= 2 * tol)
    finally:
        ctx.close()


def test_graph_replay_equals_fm_run(lib):
    ctx = lib.Context(device=0)
    try:
        wl = synth.uneven_frames(24, seed=8)
        b = Batch(lib, wl)
        ctx.run(b.frames)
        ref = b.results()
        g = ctx.graph(b.frames)
        try:
            b.clear()
            l0 = lib.fm_launch_count(ctx.h)
            g.launch()
            got = b.results()
            assert lib.fm_launch_count(ctx.h) > l0
            for (P0, i0, s0), (P1, i1, s1) in zip(ref, got):
                assert s1 == 0 and np.array_equal(P0, P1) and np.array_equal(i0, i1)
            # new inputs in the same buffers: the replay follows them
            wl2 = synth.uneven_frames(24, seed=8)
            rng = np.random.default_rng(1)
            for (X, *_), fr in zip(b.bufs, wl2.frames):
                X.copy_(torch.from_numpy((fr.X * np.exp(1j * rng.uniform(0, 6.28))).astype(np.complex64)))
            ctx.run(b.frames)
            ref2 = b.results()
            b.clear()
            g.launch()
            g.launch()  # launches on one stream run back to back
            got2 = b.results()
            for (P0, i0, s0), (P1, i1, s1) in zip(ref2, got2):
                assert np.array_equal(P0, P1) and np.array_equal(i0, i1)
        finally:
            g.close()
    finally:
        ctx.close()


def test_autotune_picks_a_working_path(lib):
    ctx = lib.Context(device=0)
    try:
        b = Batch(lib, synth.uneven_frames(16, seed=9))
        cp, sp, ms = ctx.autotune(b.frames, reps=2)
        assert cp in (lib.FM_COV_TC, lib.FM_COV_SIMT) and sp in (lib.FM_COV_TC, lib.FM_COV_SIMT) and ms > 0
        b.clear()
        ctx.run(b.frames)
        for P, idx, st in b.results():
            assert st == 0 and np.all(P > 0)
    finally:
        ctx.close()


def test_run_host_matches_device_run(lib):
    """fm_run_host (host X and outputs, strided rows) gives fm_run's results bit for bit,
    also with two calls in flight on one stream."""
    ctx = lib.Context(device=0)
    try:
        wl = synth.uneven_frames(10, seed=12)
        b = Batch(lib, wl)
        ctx.run(b.frames)
        ref = b.results()
        hosts, frames = [], []
        for fr in wl.frames:
            M, T = fr.X.shape
            Xh = torch.zeros((M, T + 3), dtype=torch.complex64).pin_memory()  # ldx = T + 3
            Xh[:, :T] = torch.from_numpy(fr.X)
            P = torch.full((fr.L,), -1.0, dtype=torch.float32).pin_memory()
            idx = torch.full((fr.K,), -7, dtype=torch.int32).pin_memory()
            deg = torch.empty(fr.K, dtype=torch.float32).pin_memory()
            n = torch.zeros(1, dtype=torch.int32).pin_memory()
            st = torch.full((1,), -1, dtype=torch.int32).pin_memory()
            hosts.append((Xh, P, idx, deg, n, st))
            frames.append(lib.Context.frame(Xh[:, :T], fr.K, fr.l, fr.t, 2, fr.theta0, fr.step, fr.L, P, idx, deg, n,
                                            seed=3, frame_id=fr.frame_id, status=st))
        ctx.run_host(frames)
        ctx.run_host(frames)  # second call overlaps the first one's chain
        torch.cuda.synchronize()
        for (P0, i0, s0), (Xh, P, idx, deg, n, st) in zip(ref, hosts):
            assert int(st.item()) == 0
            assert np.array_equal(P0, P.numpy()) and np.array_equal(i0, idx.numpy())
    finally:
        ctx.close()


def test_odd_rows_take_the_tensor_core_covariance(lib):
    """Frames whose rows TMA cannot address (odd ldx, or a base off a 16-byte boundary) are
    copied into padded rows first, so the whole uneven batch takes the tensor-core covariance;
    the result matches the CUDA-core covariance path: same peaks, and the denominator
    M - ||U_s^H a||^2 of every grid point within 1e-5 M (the projector accuracy of the FP32
    path, scaled by ||a||^2 = M; a dB bound would divide this by the near-zero denominator
    of a peak top)."""
    ctx = lib.Context(device=0)
    try:
        wl = synth.uneven_frames(12, seed=21)
        assert any(fr.X.shape[1] % 2 for fr in wl.frames)
        b = Batch(lib, wl)
        # one frame more whose X starts 8 bytes into its buffer
        fr = wl.frames[0]
        M, T = fr.X.shape
        big = torch.zeros(M * T + 1, dtype=torch.complex64, device="cuda")
        big[1:] = torch.from_numpy(np.ascontiguousarray(fr.X).ravel()).cuda()
        Xoff = big[1:].view(M, T)
        assert Xoff.data_ptr() % 16 == 8
        P = torch.full((fr.L,), -1.0, dtype=torch.float32, device="cuda")
        idx = torch.full((fr.K,), -7, dtype=torch.int32, device="cuda")
        deg = torch.empty(fr.K, dtype=torch.float32, device="cuda")
        n = torch.zeros(1, dtype=torch.int32, device="cuda")
        st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        b.bufs.append((Xoff, P, idx, deg, n, st))
        b.frames.append(lib.Context.frame(Xoff, fr.K, fr.l, fr.t, 2, fr.theta0, fr.step, fr.L, P, idx, deg, n,
                                          seed=3, frame_id=99, status=st))
        out = {}
        for path in (lib.FM_COV_SIMT, lib.FM_COV_AUTO):
            ctx.set_cov_path(path)
            b.clear()
            ctx.run(b.frames)
            out[path] = b.results()
            if path == lib.FM_COV_AUTO:
                assert ctx.last_cov_path() == lib.FM_COV_TC
        ctx.set_cov_path(lib.FM_COV_AUTO)
        Ms = [f.X.shape[0] for f in wl.frames] + [M]
        for m, (Ps, is_, ss), (Pt, it, stt) in zip(Ms, out[lib.FM_COV_SIMT], out[lib.FM_COV_AUTO]):
            assert ss == 0 and stt == 0
            assert np.array_equal(np.sort(is_), np.sort(it))
            d = np.max(np.abs(1.0 / Pt.astype(np.float64) - 1.0 / Ps.astype(np.float64)))
            assert d <= 1e-5 * m, (m, d)
    finally:
        ctx.close()

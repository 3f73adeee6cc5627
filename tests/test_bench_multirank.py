"""The N>1 bench path on CPU: two gloo ranks, as torchrun would launch them.

Frames are independent problems, so the ranks share no data: each owns a disjoint
block of frame ids and its own seeded frames, and the only collective is the
max-over-ranks of the timed region that the whole-job rate divides by."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

WORLD = 2
B = 3


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    from paper_1911_07434_gb300 import synth
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(WORLD))
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        ids = bench.shard_frame_ids(rank, B)
        wl = synth.massive_mimo_frames(B, seed=rank, M=32, T=48, K=2, extra=2, grid=(-60.0, 60.0, 1.0))
        secs = 1.0 + rank                      # rank 1 is the slower one
        slowest = bench.max_over_ranks(secs, torch.device("cpu"))
        out[rank] = {"ids": ids, "slowest": slowest, "rate": bench.job_rate(WORLD, B, 4, slowest),
                     "x00": complex(wl.frames[0].X[0, 0])}
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_frames_and_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, port, out)) for r in range(WORLD)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    ids = sorted(res[0]["ids"] + res[1]["ids"])
    assert ids == list(range(WORLD * B))                        # disjoint, covering
    assert res[0]["slowest"] == res[1]["slowest"] == 2.0         # max over ranks on every rank
    assert res[0]["rate"] == pytest.approx(WORLD * B * 4 / 2.0)  # whole-job frames/s
    assert res[0]["x00"] != res[1]["x00"]                        # each rank its own frames

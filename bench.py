#!/usr/bin/env python3
"""Benchmark: AoA frames/s of the fast-MUSIC hot path at M=512 on GB300.

Workload (one step = one fm_run over a batch): 64 synthetic ULA frames, M=512
antennas, T=1024 snapshots, K=8 sources uniform in +-60 deg (>= 2 deg apart),
per-source SNR U(0, 20) dB, l = K + 16 = 24, one power iteration, random
projection, 15001-point grid over +-75 deg (0.01 deg).  The batch's snapshots
(268 MB) exceed the 129 MB L2, so no flush is needed between steps.

Printed JSON line (rank 0): value = frames/s of the whole job with inputs
resident in HBM; e2e = the same through the C ABI with host buffers
(fm_run_host: every step's pinned-host -> device copy of X and device -> host
copy of P and the peaks inside the timed region, overlapped by the library with
the previous step's chain); roofline of the dominant kernel from CUDA events on the launching
stream; full-eig MUSIC on the same GPU (our covariance + torch.linalg.eigh +
our scan and peaks) for the speed-up; the FP64 oracle timed on the host cores
as cpu_baseline.  `--impl reference` times the oracle alone as the reference
arm (bounded sample per step).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "AoA frames/s at M=512 (fast-MUSIC vs full-eig MUSIC, same GPU); p99 latency"
UNIT = "frames/s"
BATCH = 64


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--method", default="projection", choices=["projection", "sampling"])
    ap.add_argument("--prec", default="fp32", choices=["fp32", "tf32", "bf16"],
                    help="operand precision of the covariance / sketch / scan GEMMs (FP32: three-term split products, TF32 pairs in the covariance and sketch, FP16 pairs in the scan)")
    ap.add_argument("--batch", type=int, default=BATCH)
    ap.add_argument("--no-baseline", action="store_true", help="skip full-eig MUSIC and the CPU oracle")
    ap.add_argument("--cpu-sample", type=int, default=3, help="frames of the workload the oracle times")
    ap.add_argument("--serve-requests", type=int, default=4000, help="requests of the timed serving run (0: skip)")
    ap.add_argument("--serve-rate", type=float, default=20000.0, help="Poisson arrival rate of the serving run")
    ap.add_argument("--uneven-frames", type=int, default=4096, help="frames of the uneven-batch run (0: skip)")
    ap.add_argument("--precision-frames", type=int, default=32, help="frames of the precision study (0: skip)")
    ap.add_argument("--no-variants", dest="variants", action="store_false",
                    help="skip the sampling variant and the M = 64 frame")
    ap.add_argument("--serve-sweep", default="40000,80000,160000,320000",
                    help="offered rates (frames/s) of the serving sweep, '' to skip")
    return ap.parse_args()


def workload_config(method: str, batch: int, prec: str = "fp32"):
    return {"workload": f"ULA M=512 T=1024 K=8 l=24 t=1 L=15001, {batch} frames per step",
            "method": "random projection (Alg. 2)" if method == "projection" else "random sampling (Alg. 1)",
            "frames_per_step": batch, "M": 512, "T": 1024, "K": 8, "l": 24, "t": 1, "L": 15001,
            "precision": {"fp32": "FP32 (split products on the tensor cores: 3xTF32 covariance and sketch, 3xFP16 scan)", "tf32": "TF32 operands",
                          "bf16": "BF16 operands"}[prec],
            "l2_flush": "none: inputs (268 MB/step) exceed the 129 MB L2"}


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def peaks_json():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
        "fallback"


def cpu_oracle_rate(frames, method_id, n):
    """Time the FP64 oracle (single-threaded C) on the first n frames; frames/s."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    for fr in frames[:n]:
        oracle.frame(fr.X, fr.K, fr.l, fr.t, method_id, 0, fr.frame_id, fr.theta0, fr.step, fr.L)
    dt = time.perf_counter() - t0
    return n / dt, dt


def _oracle_frame_job(job):
    """One frame through the FP64 oracle in a worker process (spawned, so it never inherits a
    CUDA context); returns the seconds it took."""
    import oracle
    if job is None:             # warm-up: load the library in this worker
        oracle.build()
        return 0.0
    X, K, l, t, method_id, fid, theta0, step, L = job
    t0 = time.perf_counter()
    oracle.frame(X, K, l, t, method_id, 0, fid, theta0, step, L)
    return time.perf_counter() - t0


def cpu_oracle_rate_parallel(frames, method_id, workers, per_worker=2):
    """The oracle as it stands, one frame per task over `workers` spawned processes on the
    host cores: frames/s over workers x per_worker frames of the workload (wall clock)."""
    import multiprocessing
    from concurrent.futures import ProcessPoolExecutor
    n = min(len(frames), workers * per_worker)
    jobs = [(fr.X, fr.K, fr.l, fr.t, method_id, fr.frame_id, fr.theta0, fr.step, fr.L) for fr in frames[:n]]
    with ProcessPoolExecutor(max_workers=workers, mp_context=multiprocessing.get_context("spawn")) as ex:
        list(ex.map(_oracle_frame_job, [None] * workers))
        t0 = time.perf_counter()
        list(ex.map(_oracle_frame_job, jobs))
        dt = time.perf_counter() - t0
    return n / dt, dt, n


def run_reference(args):
    """Reference arm: the FP64 oracle on the host cores, one frame per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_1911_07434_gb300 import synth
    method_id = 2 if args.method == "projection" else 1
    n = args.warmup + args.steps
    wl = synth.massive_mimo_frames(n, seed=0)
    import oracle
    oracle.build()
    times = []
    for i, fr in enumerate(wl.frames):
        t0 = time.perf_counter()
        oracle.frame(fr.X, fr.K, fr.l, fr.t, method_id, 0, fr.frame_id, fr.theta0, fr.step, fr.L)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    total = sum(times)
    value = len(times) / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args.method, args.batch, args.prec),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "one frame of the workload per step, single-threaded FP64 C oracle"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


TF32_PER_BF16 = 1.1 / 2.25   # nominal dense TF32 / BF16 tensor rate on GB300 (profiling recipe)


def peak_3xtf32():
    """FP32-equivalent tensor peak: measured BF16 burst x nominal TF32/BF16 ratio / 3."""
    pk, _ = peaks_json()
    return pk.get("bf16_tflops", 1895.2) * TF32_PER_BF16 / 3.0


def profile_traffic(name):
    """DRAM bytes per launch (read + write) recorded in the committed ncu summary, or None."""
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    rd = wr = None
    for line in open(path):
        cells = [c.strip() for c in line.split("|")]
        if len(cells) > 3 and cells[1] == "dram__bytes_read.sum":
            rd = float(cells[2]) * (1e6 if cells[3].lower().startswith("mbyte") else 1e9 if cells[3].lower().startswith("gbyte") else 1.0)
        if len(cells) > 3 and cells[1] == "dram__bytes_write.sum":
            wr = float(cells[2]) * (1e6 if cells[3].lower().startswith("mbyte") else 1e9 if cells[3].lower().startswith("gbyte") else 1.0)
    return (rd + wr) if rd is not None and wr is not None else None


def roofline(stages, ctx, pk, pk_kind, B, M, T, K, L, prec="fp32"):
    """Roofline entry for the covariance (the dominant contraction of the step).

    achieved = algorithmic FP32 flops per launch (4 M^2 T per frame: the Hermitian
    half of X X^H) / average launch time from CUDA events on the launching stream.
    Tensor-core path: every FP32 product costs three TF32 MMAs (3xTF32), so the
    peak is the TF32 dense peak / 3, the TF32 peak being the measured BF16 burst
    peak x the nominal TF32/BF16 ratio.  CUDA-core path: FP32 FFMA peak from the
    SM count, lanes and the measured maximum SM clock."""
    from paper_1911_07434_gb300 import binding
    cov_ms, cov_n = stages["covariance"]
    avg_s = cov_ms / max(cov_n, 1) / 1e3
    flops = 4.0 * M * M * T * B
    achieved = flops / avg_s / 1e12
    if ctx.last_cov_path() == binding.FM_COV_TC and prec != "fp32":
        bf16 = pk.get("bf16_tflops", 1895.2)
        peak = bf16 if prec == "bf16" else bf16 * TF32_PER_BF16
        return {"kernel": f"covariance (cov_tc_kernel, tcgen05, {prec.upper()} operands)", "bound": "tensor",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                "algorithmic_bytes": 8.0 * M * T * B + 8.0 * M * M * B, "avg_launch_ms": avg_s * 1e3,
                "peak_source": f"bf16_tflops {bf16} ({pk_kind})" + ("" if prec == "bf16" else
                                                                    f" x {TF32_PER_BF16:.4f} (nominal TF32/BF16)")}
    if ctx.last_cov_path() == binding.FM_COV_TC:
        tf32 = pk.get("bf16_tflops", 1895.2) * TF32_PER_BF16
        peak = tf32 / 3.0
        return {"kernel": "covariance (cov_tc_kernel, tcgen05 kind::tf32, 3xTF32)", "bound": "tensor",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "frac_of_tf32_peak": achieved / tf32,
                "traffic": profile_traffic("cov_tc_kernel_ula_M512_T1024_B64.md"),
                "algorithmic_bytes": 8.0 * M * T * B + 8.0 * M * M * B, "avg_launch_ms": avg_s * 1e3,
                "peak_source": f"TF32 = bf16_tflops {pk.get('bf16_tflops')} ({pk_kind}) x {TF32_PER_BF16:.4f}; "
                               f"/3 for three TF32 MMAs per FP32 product"}
    fp32 = 152 * 128 * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    return {"kernel": "covariance (cov_fp32_kernel)", "bound": "alu", "achieved": achieved, "peak": fp32,
            "unit": "TFLOP/s", "frac": achieved / fp32, "traffic": None, "avg_launch_ms": avg_s * 1e3,
            "peak_source": f"FP32 FFMA: 152 SMs x 128 lanes x 2 flop x sm_max_mhz ({pk_kind})"}


def shard_frame_ids(rank: int, batch: int) -> list:
    """Frames are independent problems: rank r owns frame ids [r * batch, (r + 1) * batch)."""
    return [rank * batch + b for b in range(batch)]


def max_over_ranks(x: float, device) -> float:
    """Largest value of x over the ranks of the default process group (x itself without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, batch: int, steps: int, seconds: float) -> float:
    """Whole-job frames/s: every rank ran `steps` batches of `batch` frames; `seconds` is the
    slowest rank's time."""
    return world * batch * steps / seconds


def pct(vals, q):
    """q-th percentile (0..100) of vals by the nearest-rank rule."""
    v = sorted(vals)
    return v[min(len(v) - 1, max(0, int(round(q / 100.0 * len(v) + 0.5)) - 1))]


def event_times(fn, reps, stream, warm=3):
    """Per-call device time (ms) of fn() over reps calls, CUDA events on `stream`, one
    synchronisation per call (latency, not throughput)."""
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    out = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        out.append(e0.elapsed_time(e1))
    return out


def frame_flops(M, T, K, l, t, L, method):
    """Algorithmic flops of one frame: covariance 4 M^2 T (Hermitian half), sketch
    8 M^2 l per product (t + 1 products for projection, t for sampling), scan 8 L M K."""
    prods = t + 1 if method == 2 else t
    return 4.0 * M * M * T + 8.0 * M * M * l * prods + 8.0 * L * M * K


def serving_run(binding, synth, dev, n_req, rate, budget_gb=40, pool_per_profile=8, seed=0):
    """Streaming request loop of the serving mix: Poisson arrivals at `rate` drawn equally from
    the three range profiles (long M=256 / medium M=384 / short M=512), served by
    fm_serve_submit / fm_serve_poll under a `budget_gb` workspace budget.  Latency of a request =
    time its completion is observed - its scheduled arrival time (host clock)."""
    import numpy as np
    import torch
    profiles = list(synth.SERVING_PROFILES)
    pool = []
    for pi, name in enumerate(profiles):
        for j in range(pool_per_profile):
            fr = synth.serving_frame(name, frame_id=pi * 1000 + j, seed=seed)
            pool.append((fr, torch.from_numpy(np.ascontiguousarray(fr.X)).to(dev)))
    Lmax = max(fr.L for fr, _ in pool)
    Kmax = max(fr.K for fr, _ in pool)
    rng = np.random.default_rng(seed + 77)
    n_warm = min(400, n_req)
    n_all = n_warm + n_req
    pick = [(i % 3) * pool_per_profile + int(rng.integers(pool_per_profile)) for i in range(n_all)]
    P = torch.empty((n_all, Lmax), dtype=torch.float32, device=dev)
    idx = torch.empty((n_all, Kmax), dtype=torch.int32, device=dev)
    deg = torch.empty((n_all, Kmax), dtype=torch.float32, device=dev)
    npk = torch.empty(n_all, dtype=torch.int32, device=dev)
    st = torch.zeros(n_all, dtype=torch.int32, device=dev)
    fs = []
    for i in range(n_all):
        fr, X = pool[pick[i]]
        fs.append(binding.Context.frame(X, fr.K, fr.l, fr.t, binding.FM_RAND_PROJECTION, fr.theta0, fr.step, fr.L,
                                        P[i], idx[i], deg[i], npk[i:i + 1], seed=1, frame_id=i,
                                        status=st[i:i + 1]))
    ctx = binding.Context(budget_bytes=budget_gb << 30, device=dev.index or 0)

    def stream(lo, hi, arrive):
        lat = []
        pend = []                        # (ticket, arrival) in arrival order
        i = lo
        t0 = time.perf_counter()
        while i < hi or pend:
            now = time.perf_counter() - t0
            while i < hi and arrive[i - lo] <= now:
                pend.append((ctx.serve_submit(fs[i]), arrive[i - lo]))
                i += 1
            keep = []
            for k, (tk, ta) in enumerate(pend):
                if k < 32 and ctx.serve_poll(tk):
                    lat.append(time.perf_counter() - t0 - ta)
                else:
                    keep.append((tk, ta))
            pend = keep
        return lat, time.perf_counter() - t0

    gaps = rng.exponential(1.0 / rate, size=n_all)
    stream(0, n_warm, np.cumsum(gaps[:n_warm]))
    torch.cuda.synchronize()
    l0 = binding.fm_launch_count(ctx.h)
    arrive = np.cumsum(gaps[n_warm:])
    lat, wall = stream(n_warm, n_all, arrive)
    torch.cuda.synchronize()
    launches = binding.fm_launch_count(ctx.h) - l0
    assert int(st.abs().sum()) == 0, "a served frame reported a non-zero status"
    ctx.close()
    lat = np.sort(np.asarray(lat)) * 1e3
    return {"offered_frames_per_s": rate, "frames_per_s": n_req / wall, "requests": n_req,
            "p50_ms": float(lat[len(lat) // 2]), "p99_ms": float(lat[int(0.99 * (len(lat) - 1))]),
            "max_ms": float(lat[-1]), "budget_gb": budget_gb, "gpu_launches": int(launches),
            "profiles": {k: {"M": v[0], "T": v[1], "K_max": v[2], "fov_deg": v[3], "step_deg": v[4]}
                         for k, v in synth.SERVING_PROFILES.items()},
            "latency": "observed completion - scheduled Poisson arrival (host clock, polled)"}


def uneven_run(binding, synth, dev, n_frames=4096, pool=256, steps=3, seed=0):
    """Uneven batch: n_frames frames (M in {128, 192, 256, 384, 512}, T log-uniform in
    [64, 2048], K in [1, 12], l = K + 12, t = 1, 0.05 deg grid over +-75 deg) in one fm_run,
    timed plainly, as a replayed CUDA graph, and after the path autotuner.  `pool` distinct
    frames are drawn and copied into n_frames separate device buffers."""
    import numpy as np
    import torch
    wl = synth.uneven_frames(pool, seed=seed)
    frames, bufs = [], []
    for i in range(n_frames):
        fr = wl.frames[i % pool]
        X = torch.from_numpy(np.ascontiguousarray(fr.X)).to(dev)
        P = torch.empty(fr.L, dtype=torch.float32, device=dev)
        idx = torch.empty(fr.K, dtype=torch.int32, device=dev)
        deg = torch.empty(fr.K, dtype=torch.float32, device=dev)
        npk = torch.empty(1, dtype=torch.int32, device=dev)
        st = torch.zeros(1, dtype=torch.int32, device=dev)
        bufs.append((X, P, idx, deg, npk, st))
        frames.append(binding.Context.frame(X, fr.K, fr.l, fr.t, binding.FM_RAND_PROJECTION, fr.theta0, fr.step,
                                            fr.L, P, idx, deg, npk, seed=1, frame_id=i, status=st))
    ctx = binding.Context(device=dev.index or 0)
    stream = torch.cuda.current_stream()

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps, (time.perf_counter() - t0) * 1e3 / steps

    run_ms, run_wall = timed(lambda: ctx.run(frames))
    l0 = ctx.launch_count()
    ctx.stage_times(reset=True)
    ctx.set_timing(True)
    ctx.run(frames)
    ctx.set_timing(False)
    stg = ctx.stage_times(reset=True)
    per_run = ctx.launch_count() - l0
    cov, scan, tuned_ms = ctx.autotune(frames, reps=2)
    run2_ms, _ = timed(lambda: ctx.run(frames))
    t0 = time.perf_counter()
    g = ctx.graph(frames)
    create_s = time.perf_counter() - t0
    graph_ms, graph_wall = timed(g.launch)
    g.close()
    bad = sum(int(b[5].abs().sum().item()) != 0 for b in bufs)
    ctx.close()
    names = {binding.FM_COV_TC: "tensor", binding.FM_COV_SIMT: "cuda-core"}
    flops = sum(frame_flops(f.M, f.T, f.K, f.l, f.t, f.L, 2) for f in (wl.frames[i % pool] for i in range(n_frames)))
    best_ms = min(run_ms, run2_ms, graph_ms)
    tf = flops / (best_ms / 1e3) / 1e12
    return {"frames": n_frames, "distinct_frames": pool, "gpu_launches_per_step": int(per_run),
            "algorithmic_tflop_per_step": flops / 1e12,
            "roofline": {"bound": "tensor", "achieved": tf, "unit": "TFLOP/s",
                         "peak": peak_3xtf32(), "frac": tf / peak_3xtf32(),
                         "note": "covariance + sketch + scan flops of the batch over its best step time "
                                 "(fm_run, autotuned or graph replay); peak = the 3xTF32 peak of the headline"},
            "stage_ms": {k: round(v[0], 4) for k, v in stg.items() if v[1]},
            "fm_run": {"frames_per_s": n_frames / (run_ms / 1e3), "ms_per_step": run_ms,
                       "host_wall_ms_per_step": run_wall},
            "autotuned": {"covariance": names.get(cov), "scan": names.get(scan),
                          "frames_per_s": n_frames / (run2_ms / 1e3), "ms_per_step": run2_ms},
            "cuda_graph": {"frames_per_s": n_frames / (graph_ms / 1e3), "ms_per_step": graph_ms,
                           "host_wall_ms_per_step": graph_wall, "create_s": create_s},
            "frames_with_nonzero_status": bad}


def precision_run(binding, synth, dev, n_frames=32, steps=3, seed=0):
    """Precision study (M=1024, T=2048, K=16, l=48, t=1, 36001-point grid, 32 frames): frames/s
    of each precision mode with and without the FP32 refinement step, and each mode's distance
    to the all-FP32 run on the same frames (projector ||U U^H - U32 U32^H||_F, max over frames;
    peak indices equal)."""
    import numpy as np
    import torch
    wl = synth.precision_study_frames(n_frames, seed=seed)
    f0 = wl.frames[0]
    M, T = f0.X.shape
    K, l, t, L = f0.K, f0.l, f0.t, f0.L
    X = torch.from_numpy(np.stack([f.X for f in wl.frames])).to(dev)
    P = torch.empty((n_frames, L), dtype=torch.float32, device=dev)
    idx = torch.empty((n_frames, K), dtype=torch.int32, device=dev)
    deg = torch.empty((n_frames, K), dtype=torch.float32, device=dev)
    npk = torch.empty(n_frames, dtype=torch.int32, device=dev)
    st = torch.zeros(n_frames, dtype=torch.int32, device=dev)
    ctx = binding.Context(device=dev.index or 0)
    stream = torch.cuda.current_stream()
    out, ref = {}, None
    names = {binding.FM_PREC_FP32: "fp32", binding.FM_PREC_TF32: "tf32", binding.FM_PREC_BF16: "bf16"}
    for prec in (binding.FM_PREC_FP32, binding.FM_PREC_TF32, binding.FM_PREC_BF16):
        for refine in (0, 1):
            fs = [ctx.frame(X[b], K, l, t, binding.FM_RAND_PROJECTION, f0.theta0, f0.step, L, P[b], idx[b], deg[b],
                            npk[b:b + 1], seed=1, frame_id=wl.frames[b].frame_id, status=st[b:b + 1], prec=prec,
                            refine=refine) for b in range(n_frames)]
            ctx.run(fs)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                ctx.run(fs)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            U = [ctx.run_subspace(b, M, K).cpu().numpy().astype(np.complex128) for b in range(n_frames)]
            pk = np.sort(idx.cpu().numpy(), axis=1)
            r = {"frames_per_s": n_frames / (ms / 1e3), "ms_per_step": ms, "status_ok": int(st.abs().sum()) == 0}
            if ref is None:
                ref = (U, pk)
            else:
                r["proj_vs_fp32"] = max(float(np.linalg.norm(u @ u.conj().T - v @ v.conj().T)) for u, v in zip(U, ref[0]))
                r["peaks_equal_fp32"] = bool(np.array_equal(pk, ref[1]))
            out[f"{names[prec]}{'+refine' if refine else ''}"] = r
    ctx.close()
    return {"workload": wl.name, "frames": n_frames, "modes": out}


def variants_run(binding, synth, ctx, X, B, M, T, K, l, L, fr0, wl, dev, stream, steps):
    """The headline workload's other forms: random sampling (Alg. 1, t = 0) and random
    sampling with the FP32 refinement step, each as a 64-frame batch and as single
    frames; and the M = 64 frame (K = 3, T = 200, l = 13, t = 2, 1801 angles) with random
    projection and with standard MUSIC.  Device-timed with CUDA events; U_s of frame 0
    of each kept for the accuracy check of the CPU leg."""
    import numpy as np
    import torch
    from paper_1911_07434_gb300.full_eig import full_eig_music
    out = {}
    P = torch.empty((B, L), dtype=torch.float32, device=dev)
    idx = torch.empty((B, K), dtype=torch.int32, device=dev)
    deg = torch.empty((B, K), dtype=torch.float32, device=dev)
    npk = torch.empty(B, dtype=torch.int32, device=dev)
    st = torch.zeros(B, dtype=torch.int32, device=dev)
    for name, t_, refine in (("sampling_t0", 0, 0), ("sampling_t0_refine", 0, 1)):
        fs = [ctx.frame(X[b], K, l, t_, binding.FM_RAND_SAMPLING, fr0.theta0, fr0.step, L, P[b], idx[b], deg[b],
                        npk[b:b + 1], seed=0, frame_id=wl.frames[b].frame_id, status=st[b:b + 1], refine=refine)
              for b in range(B)]
        batch = event_times(lambda: ctx.run(fs), max(10, steps), stream)
        ctx.set_timing(True)
        ctx.run(fs)
        ctx.set_timing(False)
        stg = ctx.stage_times(reset=True)
        tot = sum(v[0] for v in stg.values()) or 1.0
        U0 = ctx.run_subspace(0, M, K).cpu().numpy()
        one = event_times(lambda: ctx.run(fs[:1]), 30, stream)
        ok = int(st.abs().sum()) == 0
        out[name] = {"method": "random sampling (Alg. 1)" + (" + FP32 refinement step" if refine else ""),
                     "t": t_, "refine": refine, "frames_per_s": B / (statistics.mean(batch) / 1e3),
                     "step_ms": {"p50": pct(batch, 50), "p99": pct(batch, 99)},
                     "single_frame_ms": {"p50": pct(one, 50), "p99": pct(one, 99)},
                     "stage_share": {k: round(v[0] / tot, 4) for k, v in stg.items() if v[1]},
                     "status_ok": ok, "_U0": U0}
    # the M = 64 frame: random projection and standard MUSIC, one frame per call
    sf = synth.small_frame()
    Xs = torch.from_numpy(sf.X).to(dev)
    Ps = torch.empty(sf.L, dtype=torch.float32, device=dev)
    i_s = torch.empty(sf.K, dtype=torch.int32, device=dev)
    d_s = torch.empty(sf.K, dtype=torch.float32, device=dev)
    n_s = torch.empty(1, dtype=torch.int32, device=dev)
    s_s = torch.zeros(1, dtype=torch.int32, device=dev)
    f = [ctx.frame(Xs, sf.K, sf.l, sf.t, binding.FM_RAND_PROJECTION, sf.theta0, sf.step, sf.L, Ps, i_s, d_s, n_s,
                   seed=0, frame_id=0, status=s_s)]
    proj_ms = event_times(lambda: ctx.run(f), 50, stream)
    U0 = ctx.run_subspace(0, sf.M, sf.K).cpu().numpy()
    full_ms = event_times(lambda: full_eig_music(ctx, Xs, sf.K, sf.theta0, sf.step, sf.L), 50, stream)
    out["small_frame_M64"] = {
        "workload": "ULA M=64 T=200 K=3 (-20, 5, 30 deg) 10 dB, l=13, t=2, L=1801, one frame per call",
        "projection": {"frames_per_s": 1e3 / statistics.mean(proj_ms), "p50_ms": pct(proj_ms, 50),
                       "p99_ms": pct(proj_ms, 99), "peaks_deg": sorted(d_s.cpu().tolist()),
                       "status_ok": int(s_s.item()) == 0, "_U0": U0},
        "full_eig_music": {"frames_per_s": 1e3 / statistics.mean(full_ms), "p50_ms": pct(full_ms, 50),
                           "p99_ms": pct(full_ms, 99)},
        "p99_speedup_projection_vs_full": pct(full_ms, 99) / pct(proj_ms, 99)}
    return out


def variants_accuracy(variants, wl, small):
    """Projector distance ||U U^H - U_o U_o^H||_F of frame 0 of each variant to the FP64
    oracle's subspace from the same X, Omega / I (part of the CPU-baseline leg: the only
    place the benchmark runs the oracle)."""
    import numpy as np
    import oracle
    fr = wl.frames[0]
    R = oracle.covariance(fr.X)
    res = {}
    for name, t_ in (("sampling_t0", 0), ("sampling_t0_refine", 1)):
        v = variants.get(name)
        if not v:
            continue
        Uo, _, _ = oracle.fast_music(R, fr.K, fr.l, t_, oracle.SAMPLING, 0, fr.frame_id)
        U = v.pop("_U0").astype(np.complex128)
        v["projector_vs_oracle"] = float(np.linalg.norm(U @ U.conj().T - Uo @ Uo.conj().T))
        if t_ == 1:
            v["projector_note"] = "against the oracle with t + 1 power steps (the refinement step is one more)"
    sm = variants.get("small_frame_M64")
    if sm:
        Rs = oracle.covariance(small.X)
        Uo, _, _ = oracle.fast_music(Rs, small.K, small.l, small.t, oracle.PROJECTION, 0, 0)
        U = sm["projection"].pop("_U0").astype(np.complex128)
        sm["projection"]["projector_vs_oracle"] = float(np.linalg.norm(U @ U.conj().T - Uo @ Uo.conj().T))
    return res


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1911_07434_gb300 import binding, build, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()

    method_id = binding.FM_RAND_PROJECTION if args.method == "projection" else binding.FM_RAND_SAMPLING
    B = args.batch
    wl = synth.massive_mimo_frames(B, seed=rank)           # each rank: its own frames (weak scaling)
    for fr, fid in zip(wl.frames, shard_frame_ids(rank, B)):
        fr.frame_id = fid
    M, T, K, l, t, L = 512, 1024, 8, 24, 1, 15001
    fr0 = wl.frames[0]
    Xh = torch.from_numpy(np.stack([fr.X for fr in wl.frames])).pin_memory()
    X = Xh.to(dev)
    P = torch.empty((B, L), dtype=torch.float32, device=dev)
    idx = torch.empty((B, K), dtype=torch.int32, device=dev)
    deg = torch.empty((B, K), dtype=torch.float32, device=dev)
    npk = torch.empty(B, dtype=torch.int32, device=dev)
    status = torch.zeros(B, dtype=torch.int32, device=dev)
    ctx = binding.Context(device=local)
    prec_id = {"fp32": binding.FM_PREC_FP32, "tf32": binding.FM_PREC_TF32, "bf16": binding.FM_PREC_BF16}[args.prec]
    frames = [ctx.frame(X[b], K, l, t, method_id, fr0.theta0, fr0.step, L, P[b], idx[b], deg[b], npk[b:b + 1],
                        seed=0, frame_id=wl.frames[b].frame_id, status=status[b:b + 1], prec=prec_id)
              for b in range(B)]
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()

    # ---- device-resident timing -------------------------------------------------
    for _ in range(args.warmup):
        ctx.run(frames)
    torch.cuda.synchronize()
    assert int(status.abs().sum()) == 0, "a frame reported a non-zero status"
    # the timed region brackets the covariance stage only (its events give the roofline's
    # kernel duration); the per-stage breakdown comes from a short loop after it
    ctx.stage_times(reset=True)
    ctx.set_timing_mask(1 << binding.STAGES.index("covariance"))
    launches0 = ctx.launch_count()
    step_ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    step_ev[0].record(stream)
    for k in range(args.steps):
        ctx.run(frames)
        step_ev[k + 1].record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ctx.set_timing(False)
    launches = ctx.launch_count() - launches0
    paths = {"covariance": "tensor" if ctx.last_cov_path() == binding.FM_COV_TC else "cuda-core",
             "scan": {binding.FM_COV_TC: "tensor", binding.FM_COV_SIMT: "cuda-core"}.get(ctx.last_scan_path(), "mixed"),
             "sketch": {binding.FM_COV_TC: "tensor", binding.FM_COV_SIMT: "cuda-core"}.get(ctx.last_sketch_path(), "mixed")}
    step_ms = [step_ev[k].elapsed_time(step_ev[k + 1]) for k in range(args.steps)]
    total_ms = step_ev[0].elapsed_time(step_ev[-1])
    cov_timed = ctx.stage_times(reset=True)["covariance"]
    total_ms = max_over_ranks(total_ms, dev)
    value = job_rate(world, B, args.steps, total_ms / 1e3)
    # per-stage breakdown (every stage bracketed), outside the timed region
    ctx.set_timing(True)
    for _ in range(max(5, min(args.steps, 20))):
        ctx.run(frames)
    torch.cuda.synchronize()
    ctx.set_timing(False)
    stages = ctx.stage_times(reset=True)
    stages_cov_breakdown = stages["covariance"]
    stages["covariance"] = cov_timed  # the roofline uses the timed region's launches
    # the same step replayed through the library's CUDA graph of the chain (fm_graph_*)
    graph = ctx.graph(frames)
    for _ in range(3):
        graph.launch(stream)
    torch.cuda.synchronize()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    for _ in range(args.steps):
        graph.launch(stream)
    g1.record(stream)
    torch.cuda.synchronize()
    graph_ms = max_over_ranks(g0.elapsed_time(g1) / args.steps, dev)
    graph.close()
    assert int(status.abs().sum()) == 0, "a frame reported a non-zero status"

    # ---- end-to-end through the C ABI with host buffers (fm_run_host) ----------
    # Every step copies its X from pinned host memory and its P and peaks back;
    # the library overlaps the copies of one step with the chain of the previous one.
    Ph = torch.empty((B, L), dtype=torch.float32).pin_memory()
    idxh = torch.empty((B, K), dtype=torch.int32).pin_memory()
    degh = torch.empty((B, K), dtype=torch.float32).pin_memory()
    npkh = torch.empty(B, dtype=torch.int32).pin_memory()
    sth = torch.zeros(B, dtype=torch.int32).pin_memory()
    frames_h = [ctx.frame(Xh[b], K, l, t, method_id, fr0.theta0, fr0.step, L, Ph[b], idxh[b], degh[b],
                          npkh[b:b + 1], seed=0, frame_id=wl.frames[b].frame_id, status=sth[b:b + 1], prec=prec_id)
                for b in range(B)]
    e2e_steps = max(10, args.steps)
    for _ in range(2):
        ctx.run_host(frames_h, stream)
    torch.cuda.synchronize()
    assert int(sth.abs().sum()) == 0 and np.array_equal(idxh.numpy(), idx.cpu().numpy()), "host run differs"
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ctx.run_host(frames_h, stream)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, dev)
    e2e_value = job_rate(world, B, e2e_steps, e2e_s)
    h2d = Xh.numel() * Xh.element_size()
    d2h = (Ph.numel() + idxh.numel() + degh.numel() + npkh.numel() + sth.numel()) * 4

    # ---- roofline of the dominant kernel ----------------------------------------
    pk, pk_kind = peaks_json()
    names = list(stages.keys())
    roof = roofline(stages, ctx, pk, pk_kind, B, M, T, K, L, args.prec)
    tot = max(1e-9, sum(v[0] for v in stages.values()))
    stage_summary = {n: {"ms_per_launch": (stages[n][0] / stages[n][1]) if stages[n][1] else 0.0,
                         "launches": stages[n][1], "share": stages[n][0] / tot} for n in names}
    if stages_cov_breakdown[1]:  # covariance share from the same breakdown loop as the others
        tot_b = tot - stages["covariance"][0] + stages_cov_breakdown[0]
        for n in names:
            own = stages_cov_breakdown if n == "covariance" else stages[n]
            stage_summary[n]["share"] = own[0] / max(1e-9, tot_b)
    dom = max(names, key=lambda n: stage_summary[n]["share"])

    # ---- single-frame latency (one fm_run per frame, device-resident) ----------
    lat = []
    one = frames[:1]
    for _ in range(5):
        ctx.run(one)
    torch.cuda.synchronize()
    for _ in range(max(20, args.steps)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.run(one)
        e1.record(stream)
        e1.synchronize()
        lat.append(e0.elapsed_time(e1))
    lat.sort()
    single = {"p50_ms": lat[len(lat) // 2], "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
              "frames_per_s": 1e3 / lat[len(lat) // 2]}

    # ---- full-eig MUSIC on the same GPU -----------------------------------------
    full = None
    if not args.no_baseline:
        from paper_1911_07434_gb300.full_eig import full_eig_music
        batch_ms = event_times(lambda: full_eig_music(ctx, X, K, fr0.theta0, fr0.step, L), 20, stream, warm=2)
        one_ms = event_times(lambda: full_eig_music(ctx, X[:1], K, fr0.theta0, fr0.step, L), 30, stream)
        fms = statistics.mean(batch_ms)
        full = {"value": B / (fms / 1e3), "unit": UNIT, "ms_per_step": fms,
                "step_ms": {"p50": pct(batch_ms, 50), "p99": pct(batch_ms, 99), "repeats": len(batch_ms)},
                "single_frame_ms": {"p50": pct(one_ms, 50), "p99": pct(one_ms, 99), "repeats": len(one_ms)},
                "method": "standard MUSIC (Eq. 4-6): our covariance kernel + torch.linalg.eigh (cuSOLVER) + our "
                          "scan/peaks (paper_1911_07434_gb300.full_eig)",
                "speedup_fast_vs_full": (value / world) / (B / (fms / 1e3)),
                "p99_speedup_single_frame": pct(one_ms, 99) / single["p99_ms"],
                "p99_speedup_step": pct(batch_ms, 99) / pct(step_ms, 99)}

    # ---- the other workloads of the headline: sampling variant, the M = 64 frame ---
    variants = None
    if args.variants:
        variants = variants_run(binding, synth, ctx, X, B, M, T, K, l, L, fr0, wl, dev, stream, args.steps)

    # ---- serving mix: continuous batching under Poisson arrivals ----------------
    serving = None
    if args.serve_requests > 0:
        serving = serving_run(binding, synth, dev, args.serve_requests, args.serve_rate)
        sweep, limit = [], None
        for r in [float(x) for x in args.serve_sweep.split(",") if x.strip()]:
            sv = serving_run(binding, synth, dev, 2000, r)
            sweep.append({k: sv[k] for k in ("offered_frames_per_s", "frames_per_s", "p50_ms", "p99_ms")})
            if sv["p99_ms"] > 2.0 and limit is None:
                limit = r
        serving["sweep"] = sweep
        serving["p99_bound_ms"] = 2.0
        serving["first_rate_over_bound"] = limit

    # ---- uneven batch: one fm_run, CUDA graph replay, autotuned paths -----------
    uneven = None
    if args.uneven_frames > 0:
        uneven = uneven_run(binding, synth, dev, args.uneven_frames)

    # ---- precision study: TF32 / BF16 operands, FP32 refinement -------------------
    precision = None
    if args.precision_frames > 0:
        precision = precision_run(binding, synth, dev, args.precision_frames)

    # ---- CPU oracle baseline -----------------------------------------------------
    cpu = None
    if not args.no_baseline and rank == 0:
        rate1, secs1 = cpu_oracle_rate(wl.frames, method_id, args.cpu_sample)
        workers = max(1, min(os.cpu_count() or 1, 32))
        rate, secs, nfr = cpu_oracle_rate_parallel(wl.frames, method_id, workers)
        cpu = {"value": rate, "unit": UNIT, "cores": workers, "kind": "oracle",
               "sample": f"{nfr} frames of the workload through the FP64 C oracle, one frame per process on "
                         f"{workers} host cores ({secs:.1f} s wall)",
               "single_thread": {"value": rate1, "frames": args.cpu_sample, "seconds": secs1}}
        if variants:
            variants_accuracy(variants, wl, synth.small_frame())

    if variants:  # U_s kept for the accuracy check are not part of the report
        for v in variants.values():
            for sub in (v, v.get("projection", {})):
                sub.pop("_U0", None)
    srt = sorted(step_ms)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": {"fp32": "f32", "tf32": "tf32", "bf16": "bf16"}[args.prec],
        "data": "synthetic",
        "config": workload_config(args.method, B, args.prec),
        "latency_ms": {"p50_step": srt[len(srt) // 2], "p99_step": srt[min(len(srt) - 1, int(0.99 * len(srt)))],
                       "single_frame": single},
        "kernel_paths": paths,
        "cuda_graph": {"value": job_rate(world, B, 1, graph_ms / 1e3), "unit": UNIT, "ms_per_step": graph_ms,
                       "launch": "fm_graph_launch: the same chain replayed from one CUDA graph"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "roofline": roof, "dominant_stage": dom, "stages": stage_summary,
        "serving": serving, "uneven_batch": uneven, "precision_study": precision, "full_eig_music": full,
        "variants": variants, "cpu_baseline": cpu, "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

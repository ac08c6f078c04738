"""Benchmark: exact linear-memory DTW alignment on B300, in GCUPS.

Workload (default): the integer bit-exact pair -- 1-D int32 sequences, M=20000,
N=24000, values uniform in [0,255], Y a seeded monotone warp of X plus integer
noise in [-8,8]; cost |x-y|; canonical path (DIAG > UP > LEFT).  One step is one
complete alignment (every recursion level, base cases, path assembly).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints ONE JSON line.  value = problem cells (M*N, summed over ranks) per second
of device time, measured with CUDA events on the library's stream, with L2
flushed between steps (outside the events).  e2e = the same metric through the
public API with pinned host buffers (host->device copy of X, Y and device->host
copy of the path inside the timed region).  The reference arm times the CPU
oracle (textbook DTW, FP64/int64, single thread) on the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2008_02734_b300 import synth  # noqa: E402

WORKLOADS = {
    # name -> (description, M, N)
    "int_pair": ("integer bit-exact pair: int32 |x-y|, M=20000, N=24000, values U[0,255], "
                 "Y = monotone warp of X + U{-8..8}", 20000, 24000),
    "plain_float": ("plain float pair: 2000 x 12-d chroma-like FP32 vs 2500-frame warp + N(0,0.05^2), "
                    "Euclidean cost, FP64 accumulation", 2000, 2500),
}
METRIC = "GCUPS for exact linear-memory DTW alignment vs plain GPU form; p50/p99 latency"


def make_inputs(name: str, seed_offset: int = 0, size=None):
    """The workload's pair; ``size`` = (M, N) resizes it (same generator and
    seed; for profiling runs on smaller cases)."""
    if name == "int_pair":
        if size:
            return synth.int_pair(1 + seed_offset, size[0], size[1])
        return synth.workload_int_pair(seed=1 + seed_offset)
    if size:
        return synth.chroma_pair(0 + seed_offset, size[0], size[1])
    return synth.workload_plain_float(seed=0 + seed_offset)


def parse_size(text):
    if not text:
        return None
    m, n = text.lower().split("x")
    return int(m), int(n)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"sm_max_mhz": 2032.0, "hbm_gbs": 6400.0}, "fallback"


SWEEP_SRC = [os.path.join(ROOT, "paper_2008_02734_b300", "csrc", f) for f in ("sweep.cu", "dtw_common.cuh")]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "sweep_kernel_int_pair_traffic.json")


def sweep_traffic():
    """DRAM bytes per sweep launch from the committed ncu capture, or None when
    the capture is missing or the sweep kernel's source changed since it was taken."""
    import hashlib
    try:
        with open(TRAFFIC_FILE) as f:
            rec = json.load(f)
        h = hashlib.sha256()
        for src in SWEEP_SRC:
            with open(src, "rb") as f:
                h.update(f.read())
        sha = h.hexdigest()
    except (OSError, ValueError):
        return None, "no capture"
    if rec.get("source_sha256") != sha:
        return None, "kernel changed since the capture"
    return rec.get("dram_bytes_per_launch"), rec.get("command", "")


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        # raw samples: DTW_CLOCKS_DIR if set (to keep them), else the temp directory
        import tempfile
        d = os.environ.get("DTW_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, f"dtw_clocks_rank{gpu_index}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.25)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_oracle_baseline(name: str, budget_s: float = 20.0):
    """Oracle 1 (textbook DTW, single thread) on whole pairs of the workload until
    about budget_s seconds have been spent; GCUPS over the pairs run."""
    import oracle
    X, Y = make_inputs(name)
    cells, spent, runs = 0, 0.0, 0
    while spent < budget_s or runs == 0:
        t = time.perf_counter()
        oracle.dtw(X, Y)
        spent += time.perf_counter() - t
        cells += len(X) * len(Y)
        runs += 1
        if spent > budget_s / 2 and runs >= 1 and spent + spent / runs > budget_s:
            break
    return {"value": cells / spent / 1e9, "unit": "GCUPS", "cores": 1, "kind": "oracle",
            "sample": f"{runs} whole {len(X)}x{len(Y)} pair(s) through oracle 1 (textbook DTW with "
                      f"backpointers, {'int64' if X.dtype == np.int32 else 'FP64'}), {spent:.1f} s"}


def _oracle_pair_timed(name: str):
    """One whole pair of the workload through oracle 1 in this process: (wall-clock
    start, end, cells).  Runs in a spawned worker of cpu_oracle_all_cores."""
    import oracle
    X, Y = make_inputs(name)
    t0 = time.time()
    oracle.dtw(X, Y)
    return t0, time.time(), len(X) * len(Y)


def cpu_oracle_all_cores(name: str, max_workers: int = 64):
    """Oracle 1 (unchanged, single-threaded) on the host's cores at once: one whole
    pair of the workload per spawned process; GCUPS = all cells over the span from
    the first start to the last end (the host's aggregate throughput)."""
    import multiprocessing as mp
    n = max(1, min(os.cpu_count() or 1, max_workers))
    with mp.get_context("spawn").Pool(n) as pool:
        res = pool.map(_oracle_pair_timed, [name] * n)
    span = max(r[1] for r in res) - min(r[0] for r in res)
    cells = sum(r[2] for r in res)
    return {"value": cells / span / 1e9, "unit": "GCUPS", "cores": n, "kind": "oracle",
            "sample": f"{n} whole pairs of the workload through oracle 1, one per process (spawned), "
                      f"concurrently; {span:.1f} s from the first start to the last end; host has "
                      f"{os.cpu_count()} logical CPUs"}


def max_over_ranks(x: float, device) -> float:
    """The largest x over all ranks: the whole job's time is its slowest rank's."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gcups(cells_per_rank: float, ranks: int, steps: int, total_ms: float) -> float:
    """Cells of every rank's steps over the slowest rank's time (replicas: weak scaling)."""
    return ranks * cells_per_rank * steps / (total_ms / 1e3) / 1e9


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    X, Y = make_inputs(args.workload)
    M, N = len(X), len(Y)
    for _ in range(args.warmup):
        oracle.dtw(X, Y)
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        oracle.dtw(X, Y)
        times.append(time.perf_counter() - t)
    total = sum(times)
    value = M * N * args.steps / total / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GCUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "config": {"workload": WORKLOADS[args.workload][0], "M": M, "N": N},
            "cpu_baseline": {"value": value, "unit": "GCUPS", "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} whole {M}x{N} pairs through oracle 1 (single thread)"},
            "e2e": {"value": value, "unit": "GCUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "latency_ms": {"p50": 1e3 * float(np.percentile(times, 50)), "p99": 1e3 * float(np.percentile(times, 99))}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2008_02734_b300 as dtw

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    if args.no_graph:
        dtw.set_option(dtw.OPT_GRAPH, 0)
    tuned = None
    if args.variant is not None:
        dtw.set_option(dtw.OPT_SWEEP_VARIANT, args.variant)
    if args.base_area is not None:
        dtw.set_option(dtw.OPT_BASE_AREA, args.base_area)
    if args.workload == "int_pair" and not args.no_tune and args.variant is None and args.base_area is None:
        # the library's autotuner picks the lane block and the base-case cutoff for this size
        from paper_2008_02734_b300 import autotune
        tuned = autotune.tune(WORKLOADS["int_pair"][1], WORKLOADS["int_pair"][2], reps=3)
    size = parse_size(args.size)
    X, Y = make_inputs(args.workload, seed_offset=rank, size=size)
    M, N = len(X), len(Y)
    Xd = torch.from_numpy(X).to(dev)
    Yd = torch.from_numpy(Y).to(dev)
    path = torch.empty((M + N - 1, 2), dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 126 MB L2

    def step():
        return dtw.align(Xd, Yd, path_out=path)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()

    # timed steps: the production path (the level loop as one CUDA graph)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches = 0
    host_ms = []
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            t = time.perf_counter()
            _, cost = step()
            host_ms.append(1e3 * (time.perf_counter() - t))
            ev[k][1].record(stream)
            launches += dtw.get_stats()["kernel_launches"]
        torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    # roofline pass (not timed above): per-level events around every sweep launch
    dtw.set_option(dtw.OPT_TIMING, 1)
    sweep_ms, sweep_launches, ops, cells_proc = 0.0, 0, 0.0, 0
    sweep_cells = 0
    for k in range(args.steps):
        flush.zero_()
        step()
        st = dtw.get_stats()
        sweep_ms += st["sweep_ms"]
        sweep_launches += st["sweep_launches"]
        tagged = st["tag_cells"]
        ops += 5.0 * (st["sweep_cells"] - tagged) + 7.0 * tagged
        cells_proc += st["sweep_cells"] + st["base_cells"]
        sweep_cells += st["sweep_cells"]
    torch.cuda.synchronize()
    dtw.set_option(dtw.OPT_TIMING, 0)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total = max_over_ranks(sum(step_ms), dev)
    value = whole_job_gcups(M * N, ws, args.steps, total)

    # end to end: pinned host inputs and outputs through the same public call
    Xh = torch.from_numpy(X).pin_memory()
    Yh = torch.from_numpy(Y).pin_memory()
    Ph = torch.empty((M + N - 1, 2), dtype=torch.int32).pin_memory()
    dtw.align(Xh, Yh, path_out=Ph)
    e2e_ms = []
    Kh = 0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        p, c = dtw.align(Xh, Yh, path_out=Ph)
        e2e_ms.append(1e3 * (time.perf_counter() - t))
        Kh = p.shape[0]
    e2e_total = max_over_ranks(sum(e2e_ms), dev)
    e2e_value = whole_job_gcups(M * N, ws, args.steps, e2e_total)

    # the paper's plain FP64 GPU form on the same pair (one warm-up run, then the
    # mean of two timed runs on the host clock around synchronised calls)
    plain = None
    if not args.no_plain:
        pp, pc = dtw.align(Xd, Yd, plain=True)
        pts = []
        for _ in range(2):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            pp, pc = dtw.align(Xd, Yd, plain=True)
            torch.cuda.synchronize()
            pts.append(time.perf_counter() - t0)
        pt = float(np.mean(pts))
        plain = {"gcups": M * N / pt / 1e9, "ms": 1e3 * pt, "runs_ms": [1e3 * t for t in pts],
                 "cost_equal": bool(pc == cost), "warmup": 1,
                 "form": "one launch per anti-diagonal, one thread per cell, FP64 cost and DP, host recursion, "
                         "textbook DTW below side 500"}

    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return 0

    peaks, src = measured_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    clk_mhz = float(peaks.get("sm_max_mhz", 2032.0))
    peak_gops = sms * 4 * 32 * clk_mhz * 1e6 / 1e9  # one 32-lane instruction per SMSP per cycle
    achieved = ops / (sweep_ms / 1e3) / 1e9 if sweep_ms > 0 else None
    # the committed DRAM capture is of the integer pair's sweeps at the bench's size
    traffic, traffic_src = sweep_traffic() if args.workload == "int_pair" and not args.size else \
        (None, "no capture of this workload")
    if args.workload == "plain_float":
        # FP64 DP: one FP64 add per processed cell against the measured FP64-add rate
        fp64_peak = sms * FP64_ADD_PER_SM_CLK * clk_mhz * 1e6 / 1e9  # Gcells/s
        cps = sweep_cells / (sweep_ms / 1e3) / 1e9 if sweep_ms > 0 else None
        roofline = {"bound": "fp64", "kernel": "sweep_kernel", "achieved": cps, "peak": fp64_peak,
                    "unit": "Gcells/s", "frac": (cps / fp64_peak) if cps else None, "traffic": traffic,
                    "traffic_source": traffic_src,
                    "peak_source": f"{sms} SMs x {FP64_ADD_PER_SM_CLK} FP64 adds per SM and clock (measured, "
                                   f"profiles/pipe_rates.md) x {clk_mhz:.0f} MHz ({src}); one FP64 add per cell",
                    "sweep_ms_per_step": sweep_ms / args.steps, "sweep_launches_per_step": sweep_launches / args.steps,
                    "processed_cells_per_step": cells_proc / args.steps}
    else:
        roofline = None
    roofline = roofline or {"bound": "alu", "kernel": "sweep_kernel", "achieved": achieved, "peak": peak_gops,
                "unit": "Gop/s", "frac": (achieved / peak_gops) if achieved else None, "traffic": traffic,
                "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum, mean over "
                                "the sweep launches of one alignment)", "traffic_source": traffic_src,
                "peak_source": f"{sms} SMs x 4 schedulers x 32 lanes x {clk_mhz:.0f} MHz ({src} max SM clock); "
                               "op = one 32-bit lane instruction of the per-cell count (5 per cell, 7 tagged)",
                "sweep_ms_per_step": sweep_ms / args.steps, "sweep_launches_per_step": sweep_launches / args.steps,
                "processed_cells_per_step": cells_proc / args.steps}
    # the CPU baselines: rank 0 of a single-GPU run only (N > 1 runs report the GPU job)
    cpu_on = not args.no_cpu and ws == 1
    cpu = cpu_oracle_baseline(args.workload, budget_s=args.cpu_budget) if cpu_on else None
    cpu_all = cpu_oracle_all_cores(args.workload) if cpu_on else None
    disc = None
    if args.workload == "plain_float" and not args.no_cpu:
        # Section 4.3's discrepancy of the GPU path against the oracle's: float
        # costs may tie differently, so the two optimal paths need not coincide
        import oracle
        p_ref, _ = oracle.dtw(X, Y)
        err, emax = dtw.path_discrepancy(step()[0], p_ref, M, N)
        e = err.cpu().numpy().ravel()
        disc = {"of": "GPU path vs oracle 1 path", "max_frames": emax,
                "within_frames": {str(f): float(np.mean(e <= f)) for f in (0, 1, 2)}}
    # the other configurations, each with its own timing, roofline and error
    # against the oracle (single-GPU default runs of the integer pair only)
    extra = {}
    if args.workload == "int_pair" and ws == 1 and not args.no_extra:
        extra["c3_batch"] = measure_batch(steps=5, warmup=3, tune=True)
        extra["c2_precision"] = measure_precision(steps=2, warmup=3, forms=("f32cost_f64dp", "bf16cost_f32kahan"))
        extra["c4_serving"] = measure_serving(requests=2000, max_len=20000, budget_gb=64.0, rho=0.7)
    line = {
        "metric": METRIC, "value": value, "unit": "GCUPS", "n_gpus": ws, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "i32" if args.workload == "int_pair" else "f32-cost/f64-dp",
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload][0] + (f" (resized to {M} x {N})" if size else ""),
                   "M": M, "N": N, "pairs_per_rank": 1,
                   "parallelism": f"replicas{ws}", "l2": "flushed between steps (256 MiB write outside the events)",
                   "autotuned": None if tuned is None else {"sweep_variant": tuned["variant"],
                                                           "split_windows": tuned["windows"],
                                                           "base_area": tuned["base_area"],
                                                           "table": tuned["table"]},
                   "fixed": None if args.variant is None and args.base_area is None else
                   {"sweep_variant": args.variant, "base_area": args.base_area}},
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                       "host_p50": float(np.percentile(host_ms, 50))},
        "e2e": {"value": e2e_value, "unit": "GCUPS", "h2d_bytes_per_step": (M + N) * 4,
                "d2h_bytes_per_step": Kh * 8 + 8},
        "gpu_launches": launches,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "cpu_baseline_all_cores": cpu_all,
        "vs_plain_gpu": None if plain is None else {"plain": plain, "speedup": value / ws / plain["gcups"]},
        "path_discrepancy_vs_oracle": disc,
        "clocks": clk.summary(),
    }
    line.update(extra)
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


def _percentiles(ms):
    return {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99))}


# Measured per-SM-and-clock issue rates of the instructions the rooflines count
# (dtw_pipe_rates on a B300, profiles/pipe_rates.md): the FP64 add of the FP64 DP.
FP64_ADD_PER_SM_CLK = 1.65
# Algorithmic lane instructions per cell of the BF16 form: 2 adds, a maximum and a
# square root of the expanded cost, a compensated add (4) and two minima.
BF16_FORM_I_CELL = 10.0
# The FP32-cost form at d = 64 with the compensated DP: 64 lane instructions for
# the 64 differences and squares in packed FP32x2 arithmetic, a square root, and
# the compensated add and minima (10).
F32COST_D64_I_CELL = 75.0


def _peak_rates(dev=None):
    """(SM count, max SM clock in MHz, its source) of this GPU."""
    import torch
    peaks, src = measured_peaks()
    sms = torch.cuda.get_device_properties(dev or 0).multi_processor_count
    return sms, float(peaks.get("sm_max_mhz", 2032.0)), src


def _golden_rows(name):
    with open(os.path.join(ROOT, "tests", "golden", name)) as f:
        return [ln.strip().split("|") for ln in f if ln.strip() and not ln.startswith("#")]


def measure_batch(steps: int, warmup: int, tune: bool = True, check: bool = True, int_data: bool = False):
    """The uneven batch (256 chroma-like d=12 pairs; with ``int_data`` the same
    shapes with 1-D int32 |x-y| data) through dtw_align_batch: time per batch
    (CUDA events, L2 flushed between steps), GCUPS, the end-to-end figure from
    pinned host buffers, the roofline (chroma: against the FP64-add pipe, the
    FP64 DP's one add per cell; integer: against the ALU issue rate at 5
    instructions per cell) and the largest cost error against oracle 1's stored
    costs (tests/golden/batch_chroma_256.txt, batch_int_256.txt: 0 expected)."""
    import torch

    import paper_2008_02734_b300 as dtw

    pairs = synth.workload_batch_int() if int_data else synth.workload_batch()
    B = len(pairs)
    cells = float(sum(len(x) * len(y) for x, y in pairs))
    Xs = [torch.from_numpy(x).cuda() for x, _ in pairs]
    Ys = [torch.from_numpy(y).cuda() for _, y in pairs]
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    tuned = None
    if tune:
        # the library's autotuner picks the cutoff, the split windows and (integer
        # data) the lane block on this batch
        from paper_2008_02734_b300 import autotune
        tuned = autotune.tune_batch(Xs, Ys)
    for _ in range(max(warmup, 3)):
        res = dtw.align_batch(Xs, Ys)
    ms = []
    launches = 0
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        res = dtw.align_batch(Xs, Ys)
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
        launches += dtw.get_stats()["kernel_launches"]
    st = dtw.get_stats()
    processed = float(st["sweep_cells"] + st["base_cells"])
    err = None
    golden = "batch_int_256.txt" if int_data else "batch_chroma_256.txt"
    if check:
        ref = [float(r[3]) for r in _golden_rows(golden)]
        err = max(abs(c - r) / r for (_, c), r in zip(res, ref))
    # end to end from pinned host buffers (paths come back to host buffers too)
    Xh = [torch.from_numpy(x).pin_memory() for x, _ in pairs]
    Yh = [torch.from_numpy(y).pin_memory() for _, y in pairs]
    Ph = [torch.empty((len(x) + len(y) - 1, 2), dtype=torch.int32).pin_memory() for x, y in pairs]
    e2e = []
    for _ in range(max(1, steps // 2)):
        flush.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        dtw.align_batch(Xh, Yh, paths_out=Ph)
        e2e.append(1e3 * (time.perf_counter() - t))
    sms, mhz, src = _peak_rates()
    mean_ms = float(np.mean(ms))
    achieved = processed / (mean_ms / 1e3) / 1e9
    if int_data:
        peak = sms * 4 * 32 * mhz * 1e6 / 5 / 1e9  # Gcells/s at 5 lane instructions per cell
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gcells/s", "frac": achieved / peak,
                "peak_source": f"{sms} SMs x 4 schedulers x 32 lanes x {mhz:.0f} MHz ({src}) / 5 algorithmic "
                               "lane instructions per cell"}
    else:
        peak = sms * FP64_ADD_PER_SM_CLK * mhz * 1e6 / 1e9  # Gcells/s
        roof = {"bound": "fp64", "achieved": achieved, "peak": peak, "unit": "Gcells/s", "frac": achieved / peak,
                "peak_source": f"{sms} SMs x {FP64_ADD_PER_SM_CLK} FP64 adds per SM and clock (measured, "
                               f"profiles/pipe_rates.md) x {mhz:.0f} MHz ({src}); one FP64 add per processed cell"}
    data = "1-D int32 |x-y| (values U[0,255], Y = warp + U{-8..8}), int32 DP" if int_data else \
        "chroma-like d=12 FP32, FP32 cost, FP64 DP"
    return {
        "workload": f"uneven batch: {B} pairs, M log-uniform [1000,20000], N = clip(r M), "
                    f"r log-uniform [0.8,1.25]; {data}",
        "pairs": B, "problem_cells": cells, "processed_cells_per_step": processed, "steps": steps,
        "ms_per_step": mean_ms, "gcups": cells / (mean_ms / 1e3) / 1e9, "latency_ms": _percentiles(ms),
        "e2e": {"gcups": cells / (np.mean(e2e) / 1e3) / 1e9, "ms": float(np.mean(e2e)),
                "h2d_bytes_per_step": int(sum(x.nbytes + y.nbytes for x, y in pairs)),
                "d2h_bytes_per_step": int(sum(8 * (len(x) + len(y) - 1) for x, y in pairs))},
        "gpu_launches": launches, "levels": st["levels"],
        "roofline": roof,
        "max_rel_err_vs_oracle": err, "oracle_source": "tests/golden/" + golden,
        "l2": "flushed between steps",
        "autotuned": None if tuned is None else {"base_area": tuned["base_area"], "split_windows": tuned["windows"],
                                                "sweep_variant": tuned["variant"]},
    }


def run_batch_workload(args):
    """The uneven batch: 256 chroma-like d=12 pairs, M log-uniform in [1000, 20000],
    N = clip(r M), r log-uniform in [0.8, 1.25]; all pairs through dtw_align_batch
    (every pair's boxes of a level share the launches).  value = sum(M N) / time."""
    r = measure_batch(args.steps, args.warmup, tune=not args.no_tune, int_data=args.batch_data == "int")
    line = {"metric": METRIC, "value": r["gcups"], "unit": "GCUPS", "n_gpus": 1,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": r["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "i32" if args.batch_data == "int" else "f32-cost/f64-dp", "data": "synthetic",
            "config": {"workload": r["workload"], "pairs": r["pairs"], "problem_cells": r["problem_cells"],
                       "l2": r["l2"], "autotuned": r["autotuned"]},
            "latency_ms": r["latency_ms"],
            "e2e": {"value": r["e2e"]["gcups"], "unit": "GCUPS", "h2d_bytes_per_step": r["e2e"]["h2d_bytes_per_step"],
                    "d2h_bytes_per_step": r["e2e"]["d2h_bytes_per_step"]},
            "gpu_launches": r["gpu_launches"], "levels": r["levels"],
            "processed_cells_per_step": r["processed_cells_per_step"], "roofline": r["roofline"],
            "max_rel_err_vs_oracle": r["max_rel_err_vs_oracle"]}
    print(json.dumps(line), flush=True)
    return 0


GOLDEN_MFCC = os.path.join(ROOT, "tests", "golden", "mfcc_pair_60000x75000.txt")


def golden_mfcc_cost():
    """The oracle's optimal cost of the precision workload, stored by
    tests/golden/make_mfcc_pair_cost.py (oracle 2, FP64 throughout)."""
    try:
        with open(GOLDEN_MFCC) as f:
            rows = [ln.strip() for ln in f if ln.strip() and not ln.startswith("#")]
        return float(rows[-1].split("|")[3])
    except (OSError, IndexError, ValueError):
        return None


PRECISION_FORMS = (
    ("f32cost_f64dp", {}, "FP32 frame cost, FP64 DP"),
    ("f32cost_f32kahan", {"dp_f32": True}, "FP32 frame cost, compensated FP32 DP"),
    ("bf16cost_f32kahan", {"cost_bf16": True}, "BF16 tensor-core cost tiles (FP32 accumulation), compensated FP32 DP"),
)


def measure_precision(steps: int, warmup: int, forms=("f32cost_f64dp", "f32cost_f32kahan", "bf16cost_f32kahan"),
                      discrepancy: bool = True, size=None):
    """The orchestral-length pair (60000 x 64-d MFCC-like frames vs a 75000-frame
    warp plus noise) in the given precision forms: time per alignment, GCUPS,
    relative error against the FP64 oracle's stored optimum, and the roofline of
    the form's binding bound (FP64 DP: the FP64-add pipe, one add per processed
    cell; compensated FP32 forms: the ALU issue rate at the form's algorithmic
    instructions per cell).  ``size`` (M, N): a smaller pair from the same
    generator, for profiling; it has no stored optimum."""
    import torch

    import paper_2008_02734_b300 as dtw

    X, Y = synth.workload_precision() if size is None else synth.workload_precision(M=size[0], N=size[1])
    M, N = len(X), len(Y)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    stream = torch.cuda.current_stream()
    c_ref = golden_mfcc_cost() if size is None else None
    sms, mhz, src = _peak_rates()
    issue = sms * 4 * 32 * mhz * 1e6 / 1e9  # lane instructions per ns
    out, paths = {}, {}
    for name, kw, desc in PRECISION_FORMS:
        if name not in forms:
            continue
        for _ in range(max(warmup, 3)):
            dtw.align(Xd, Yd, **kw)
        ms = []
        for _ in range(steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            path, cost = dtw.align(Xd, Yd, **kw)
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        st = dtw.get_stats()
        processed = float(st["sweep_cells"] + st["base_cells"])
        mean_ms = float(np.mean(ms))
        achieved = processed / (mean_ms / 1e3) / 1e9
        if name == "f32cost_f64dp":
            rl = {"bound": "fp64", "peak": sms * FP64_ADD_PER_SM_CLK * mhz * 1e6 / 1e9,
                  "peak_source": f"{sms} SMs x {FP64_ADD_PER_SM_CLK} FP64 adds per SM and clock (measured) x "
                                 f"{mhz:.0f} MHz ({src}); one FP64 add per processed cell"}
        else:
            icell = BF16_FORM_I_CELL if name.startswith("bf16") else F32COST_D64_I_CELL
            rl = {"bound": "alu", "peak": issue / icell,
                  "peak_source": f"{sms} SMs x 4 x 32 lanes x {mhz:.0f} MHz ({src}) / {icell:.0f} algorithmic lane "
                                 "instructions per cell"}
        rl.update({"achieved": achieved, "unit": "Gcells/s", "frac": achieved / rl["peak"]})
        paths[name] = path
        out[name] = {"form": desc, "ms": mean_ms, "gcups": M * N / (mean_ms / 1e3) / 1e9, "cost": cost,
                     "rel_err_vs_oracle": None if c_ref is None else abs(cost - c_ref) / c_ref,
                     "processed_cells": processed, "roofline": rl}
    disc = None
    if discrepancy and "bf16cost_f32kahan" in paths and "f32cost_f64dp" in paths:
        # Section 4.3's alignment discrepancy of the BF16 form's path against the
        # exact form's, as the share of errors within 1, 2, 22 and 43 frames (23 ms,
        # 47 ms, 0.51 s and 1 s at the features' ~43 frames per second)
        err, emax = dtw.path_discrepancy(paths["bf16cost_f32kahan"], paths["f32cost_f64dp"], M, N)
        e = err.cpu().numpy().ravel()
        disc = {"of": "bf16cost_f32kahan path vs f32cost_f64dp path", "cells": int(err.shape[1]), "max_frames": emax,
                "within_frames": {str(f): float(np.mean(e <= f)) for f in (0, 1, 2, 22, 43)}}
    return {"workload": f"orchestral-length pair: {M} x 64-d MFCC-like vs {N}-frame warp + N(0,0.1^2)",
            "M": M, "N": N, "steps": steps, "oracle_cost": c_ref,
            "oracle_source": "tests/golden/mfcc_pair_60000x75000.txt" if size is None else None, "forms": out,
            "path_discrepancy": disc}


def run_precision_workload(args):
    """The orchestral-length pair in each precision form; value is the exact
    (FP32 cost, FP64 DP) form's GCUPS."""
    forms = tuple(args.forms.split(",")) if args.forms else ("f32cost_f64dp", "f32cost_f32kahan", "bf16cost_f32kahan")
    r = measure_precision(args.steps, args.warmup, forms=forms, size=parse_size(args.size))
    ex = r["forms"].get("f32cost_f64dp") or next(iter(r["forms"].values()))
    line = {"metric": METRIC, "value": ex["gcups"], "unit": "GCUPS", "n_gpus": 1,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ex["ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32-cost/f64-dp",
            "data": "synthetic",
            "config": {"workload": r["workload"] + "; value is the FP32-cost/FP64-DP form", "M": r["M"], "N": r["N"],
                       "oracle_cost": r["oracle_cost"], "oracle_source": r["oracle_source"]},
            "forms": r["forms"], "path_discrepancy": r["path_discrepancy"]}
    print(json.dumps(line), flush=True)
    return 0


def run_edit_workload(args):
    """Edit distance (Section 5's generalisation) through the same recursion: a
    20000-symbol sequence over 4 symbols against a 10%-mutated copy, unit costs
    (Levenshtein).  GCUPS = M N / time with device-resident inputs; e2e through
    host buffers; the edit oracle (textbook DP, one core) on the same pair as the
    CPU baseline."""
    import torch

    import oracle
    import paper_2008_02734_b300 as dtw

    X, Y = synth.workload_edit_pair()
    M, N = len(X), len(Y)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    path = torch.empty((M + N + 1, 2), dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(max(args.warmup, 3)):
        dtw.edit_align(Xd, Yd, path_out=path)
    ms, launches = [], 0
    for _ in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        _, cost = dtw.edit_align(Xd, Yd, path_out=path)
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
        launches += dtw.get_stats()["kernel_launches"]
    Xh, Yh = torch.from_numpy(X).pin_memory(), torch.from_numpy(Y).pin_memory()
    Ph = torch.empty((M + N + 1, 2), dtype=torch.int32).pin_memory()
    e2e = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        p, _ = dtw.edit_align(Xh, Yh, path_out=Ph)
        e2e.append(1e3 * (time.perf_counter() - t))
    cpu = None
    if not args.no_cpu:
        t = time.perf_counter()
        _, c_ref = oracle.edit(X, Y)
        dt = time.perf_counter() - t
        cpu = {"value": M * N / dt / 1e9, "unit": "GCUPS", "cores": 1, "kind": "oracle",
               "sample": f"one whole {M}x{N} pair through the edit oracle (textbook DP with pointers), {dt:.1f} s",
               "cost_equal": bool(c_ref == cost)}
    line = {"metric": METRIC, "value": M * N / (np.mean(ms) / 1e3) / 1e9, "unit": "GCUPS", "n_gpus": 1,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": float(np.mean(ms)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i32", "data": "synthetic",
            "config": {"workload": "edit distance: 20000 symbols over 4 vs a 10%-mutated copy, unit costs",
                       "M": M, "N": N, "cost": cost, "l2": "flushed between steps"},
            "latency_ms": _percentiles(ms),
            "e2e": {"value": M * N / (np.mean(e2e) / 1e3) / 1e9, "unit": "GCUPS", "h2d_bytes_per_step": 4 * (M + N),
                    "d2h_bytes_per_step": 8 * int(p.shape[0]) + 8},
            "gpu_launches": launches, "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)
    return 0


def run_local_workload(args):
    """Local alignment (Smith-Waterman, Section 5) in linear memory: 20000 vs 24000
    random symbols over 4 sharing a mutated 5000-symbol stretch, scores +2 / -3 /
    gap -3.  GCUPS = M N / time (three passes: end search over the whole grid,
    start search over the box before the end, global alignment of the pieces);
    the local oracle on one core as the CPU baseline."""
    import torch

    import oracle
    import paper_2008_02734_b300 as dtw

    X, Y = synth.workload_local_pair()
    M, N = len(X), len(Y)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    path = torch.empty((M + N + 1, 2), dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    sc = dict(match=2, mismatch=3, gap=3)
    for _ in range(max(args.warmup, 3)):
        dtw.local_align(Xd, Yd, path_out=path, **sc)
    ms = []
    for _ in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        p, score, se = dtw.local_align(Xd, Yd, path_out=path, **sc)
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    Xh, Yh = torch.from_numpy(X).pin_memory(), torch.from_numpy(Y).pin_memory()
    Ph = torch.empty((M + N + 1, 2), dtype=torch.int32).pin_memory()
    e2e = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        ph, _, _ = dtw.local_align(Xh, Yh, path_out=Ph, **sc)
        e2e.append(1e3 * (time.perf_counter() - t))
    cpu = None
    if not args.no_cpu:
        t = time.perf_counter()
        _, s_ref, se_ref = oracle.local(X, Y, 2, 3, 3)
        dt = time.perf_counter() - t
        cpu = {"value": M * N / dt / 1e9, "unit": "GCUPS", "cores": 1, "kind": "oracle",
               "sample": f"one whole {M}x{N} pair through the local oracle (full tables), {dt:.1f} s",
               "result_equal": bool(s_ref == score and tuple(se_ref) == tuple(se))}
    line = {"metric": METRIC, "value": M * N / (np.mean(ms) / 1e3) / 1e9, "unit": "GCUPS", "n_gpus": 1,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": float(np.mean(ms)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i32", "data": "synthetic",
            "config": {"workload": "local alignment: 20000 vs 24000 symbols over 4 sharing a 10%-mutated "
                                   "5000-symbol stretch, scores +2/-3/-3", "M": M, "N": N, "score": score,
                       "start_end": list(se), "path_nodes": int(p.shape[0]), "l2": "flushed between steps"},
            "latency_ms": _percentiles(ms),
            "e2e": {"value": M * N / (np.mean(e2e) / 1e3) / 1e9, "unit": "GCUPS", "h2d_bytes_per_step": 4 * (M + N),
                    "d2h_bytes_per_step": 8 * int(ph.shape[0]) + 48},
            "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)
    return 0


def _plain_model(samples):
    """Least-squares fit t = a L + b M N of the plain form's time per request,
    L = (M + N) max(1, log2(M N / 250000)): one launch per anti-diagonal of every
    box of the host recursion, plus the cells.  samples: (M, N, seconds)."""
    A = np.array([[(m + n) * max(1.0, math.log2(m * n / 2.5e5)), m * n] for m, n, _ in samples], dtype=np.float64)
    t = np.array([x[2] for x in samples], dtype=np.float64)
    coef, *_ = np.linalg.lstsq(A, t, rcond=None)
    return np.maximum(coef, 0.0)


def _run_stream(dtw, bufs, reqs, arrivals, bf16):
    """Submits request k at arrivals[k] seconds (all at once if arrivals is
    None), polls every request to completion; returns (makespan s, latencies ms)."""
    pend = {}
    lat = []
    t0 = time.perf_counter()
    nxt = 0
    R = len(reqs)
    while nxt < R or pend:
        now = time.perf_counter() - t0
        while nxt < R and (arrivals is None or arrivals[nxt] <= now):
            t, path, keep = dtw.submit(*bufs[nxt], cost_bf16=bf16[nxt])
            pend[t] = (time.perf_counter(), path, keep, nxt)
            nxt += 1
        for t in list(pend):
            rc, K, c = dtw.poll(t)
            if rc != dtw.PENDING:
                if rc != dtw.OK:
                    raise RuntimeError(f"request {pend[t][3]} failed: {rc}")
                lat.append(1e3 * (time.perf_counter() - pend[t][0]))
                del pend[t]
        time.sleep(5e-5)
    return time.perf_counter() - t0, lat


def measure_serving(requests: int, max_len: int, budget_gb: float, rho: float = 0.7, exact: bool = False,
                    plain_samples: int = 8, plain_budget_s: float = 8.0):
    """The serving stream (Poisson arrivals, lengths log-uniform in [500, max_len],
    d = 12 FP32-cost/FP64-DP or d = 64 BF16-cost/compensated-FP32-DP requests with
    equal probability) through dtw_submit / dtw_poll.

    1. Capacity: every request submitted at once; capacity = requests / makespan.
    2. The stream at offered load rho of that capacity (the seeded arrival
       process rescaled to rate rho x capacity): GCUPS over the makespan and the
       p50 / p99 latency from submission to result.
    3. The serial plain FP64 GPU form: timed on a seeded sample of the stream's
       requests per feature dimension (the smaller ones, within a time budget),
       fitted per dimension by t = a L + b M N, and run as a single FIFO server on
       the same arrival times (its makespan and p50 / p99 latency)."""
    import torch

    import paper_2008_02734_b300 as dtw

    dtw.set_budget(int(budget_gb * (1 << 30)))
    reqs = synth.workload_serving(R=requests, rate_hz=1.0, hi=max_len)
    feats = [r.features() for r in reqs]
    cells = float(sum(r.M * r.N for r in reqs))
    bufs = [(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()) for x, y in feats]
    torch.cuda.synchronize()
    bf16 = [r.d == 64 and not exact for r in reqs]
    # warm the engines of both groups
    for k in range(min(8, len(reqs))):
        dtw.wait(dtw.submit(*bufs[k], cost_bf16=bf16[k])[0])
    sat_s, sat_lat = _run_stream(dtw, bufs, reqs, None, bf16)
    capacity = len(reqs) / sat_s
    base = np.array([r.arrival_s for r in reqs])  # the arrival process at 1 request per second
    rate = rho * capacity
    arrivals = base / rate
    mk, lat = _run_stream(dtw, bufs, reqs, arrivals, bf16)
    # the serial plain form: a seeded sample per dimension, smallest requests first
    rng = np.random.default_rng(17)
    samples = {12: [], 64: []}
    cap_cells = {12: 5e7, 64: 2e7}  # larger requests would take seconds each in the plain form
    for dim in (12, 64):
        idx = [k for k in range(len(reqs)) if reqs[k].d == dim and reqs[k].M * reqs[k].N <= cap_cells[dim]]
        idx = sorted(rng.choice(idx, size=min(4 * plain_samples, len(idx)), replace=False),
                     key=lambda k: reqs[k].M * reqs[k].N)
        spent = 0.0
        for k in idx[:: max(1, len(idx) // plain_samples)]:
            if spent > plain_budget_s / 2:
                break
            torch.cuda.synchronize()
            t = time.perf_counter()
            dtw.align(*bufs[k], plain=True)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t
            spent += dt
            samples[dim].append((reqs[k].M, reqs[k].N, dt))
    coef = {dim: _plain_model(v) for dim, v in samples.items() if len(v) >= 2}

    def t_plain(r):
        a, b = coef[r.d]
        return a * (r.M + r.N) * max(1.0, math.log2(r.M * r.N / 2.5e5)) + b * r.M * r.N

    end = 0.0
    plat = []
    for r, at in zip(reqs, arrivals):
        end = max(end, at) + t_plain(r)
        plat.append(1e3 * (end - at))
    plain_mk = end - arrivals[0]
    return {
        "workload": f"serving stream: {len(reqs)} Poisson arrivals, lengths log-uniform [500,{max_len}], "
                    "d 12 (FP32 cost, FP64 DP) or 64 (" + ("exact form" if exact else
                    "BF16 tensor-core cost, compensated FP32 DP") + f"), admission budget {budget_gb} GB",
        "requests": len(reqs), "problem_cells": cells,
        "capacity": {"requests_per_s": capacity, "makespan_s": sat_s, "gcups": cells / sat_s / 1e9,
                     "how": "every request submitted at once"},
        "offered_load": rho, "arrival_rate_hz": rate,
        "gcups": cells / mk / 1e9, "makespan_s": mk, "latency_ms": _percentiles(lat),
        "vs_plain_gpu": {"plain_makespan_s": plain_mk, "plain_latency_ms": _percentiles(plat),
                         "makespan_speedup": plain_mk / mk,
                         "p99_ratio": float(np.percentile(plat, 99) / np.percentile(lat, 99)),
                         "how": "the plain form timed on a seeded sample per dimension, fitted by t = a (M+N) "
                                "max(1, log2(MN/250000)) + b MN, run as one FIFO server on the same arrivals",
                         "samples": {str(k): [[m, n, round(t, 4)] for m, n, t in v] for k, v in samples.items()}},
    }


def run_serving_workload(args):
    """The serving stream at offered load --rho of the capacity measured in the
    same run; value is its GCUPS."""
    r = measure_serving(args.requests, args.max_len, args.budget_gb, args.rho, args.exact)
    line = {"metric": METRIC, "value": r["gcups"], "unit": "GCUPS", "n_gpus": 1,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "mixed", "data": "synthetic",
            "config": {"workload": r["workload"], "problem_cells": r["problem_cells"], "offered_load": r["offered_load"]},
            "latency_ms": r["latency_ms"], "makespan_s": r["makespan_s"], "capacity": r["capacity"],
            "arrival_rate_hz": r["arrival_rate_hz"], "vs_plain_gpu": r["vs_plain_gpu"]}
    print(json.dumps(line), flush=True)
    return 0


def run_pipes():
    """Issue rates of the cell update's instructions on this GPU (dtw_pipe_rates),
    as thread instructions per second and per SM and clock at the measured clock,
    and the dependent-chain latencies (cycles) of the recurrence's operations."""
    import torch

    import paper_2008_02734_b300 as dtw

    torch.cuda.init()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    with ClockSampler(0) as cs:
        rates = dtw.pipe_rates()
        lat = dtw.op_latencies()
    clocks = cs.summary()
    # the measurement lasts a fraction of a second, so the median of the clock
    # samples mixes in idle readings; the kernels themselves run at the SM clock's
    # maximum (no throttle reason), which converts the rates
    mhz = clocks.get("sm_max_mhz") or measured_peaks()[0].get("sm_max_mhz", 2032.0)
    per = {k: v / (sms * mhz * 1e6) for k, v in rates.items()}
    print(json.dumps({"pipes_per_s": rates, "pipes_per_sm_clock": per, "latency_cycles": lat, "sms": sms,
                      "sm_mhz": mhz, "clocks": clocks}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["batch", "precision", "serving", "edit", "local"],
                    default="int_pair")
    ap.add_argument("--batch", type=int, default=256, help="pairs of the batch workload")
    ap.add_argument("--batch-data", choices=["chroma", "int"], default="chroma",
                    help="batch workload data: d=12 chroma-like frames (FP64 DP) or 1-D int32 |x-y|")
    ap.add_argument("--requests", type=int, default=2000, help="requests of the serving workload")
    ap.add_argument("--rho", type=float, default=0.7, help="serving workload: offered load (share of capacity)")
    ap.add_argument("--max-len", type=int, default=20000, help="longest request of the serving workload")
    ap.add_argument("--budget-gb", type=float, default=64.0, help="admission budget of the serving workload")
    ap.add_argument("--exact", action="store_true", help="serving workload: exact form for d = 64 too")
    ap.add_argument("--forms", default=None,
                    help="precision workload: comma-separated forms (f32cost_f64dp, f32cost_f32kahan, bf16cost_f32kahan)")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 GPU comparator")
    ap.add_argument("--no-extra", action="store_true",
                    help="default run: skip the batch, precision and serving configurations")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (default lane block and cutoff)")
    ap.add_argument("--variant", type=int, default=None,
                    help="integer sweep variant (lane block) to use instead of the autotuner's choice")
    ap.add_argument("--base-area", type=int, default=None,
                    help="base-case cutoff (cells) to use instead of the autotuner's choice")
    ap.add_argument("--fused-split", type=int, default=None, choices=[0, 1, 2],
                    help="where each level's split runs: 0 own launch, 1 library default, 2 in the sweep kernel")
    ap.add_argument("--size", default=None,
                    help="MxN: the pair workloads (int_pair, plain_float, precision) resized, same generator (profiling)")
    ap.add_argument("--split-windows", type=int, default=None,
                    help="windows of split rows per box and level, at most (library default 7; 1: one split row)")
    ap.add_argument("--no-graph", action="store_true",
                    help="run the level loop from the host (the same kernels; profilers list every launch)")
    ap.add_argument("--pipes", action="store_true",
                    help="measure the issue rates of the instructions the per-cell roofline counts and exit")
    args = ap.parse_args()
    if args.pipes:
        return run_pipes()
    if args.impl == "reference":
        return run_reference(args)
    if args.split_windows is not None or args.fused_split is not None:
        import paper_2008_02734_b300 as dtw
        if args.split_windows is not None:
            dtw.set_option(dtw.OPT_SPLIT_WINDOWS, args.split_windows)
        if args.fused_split is not None:
            dtw.set_option(dtw.OPT_FUSED_SPLIT, args.fused_split)
    if args.workload != "int_pair" and (args.no_graph or args.base_area is not None):
        import paper_2008_02734_b300 as dtw
        if args.no_graph:
            dtw.set_option(dtw.OPT_GRAPH, 0)
        if args.base_area is not None:
            dtw.set_option(dtw.OPT_BASE_AREA, args.base_area)
    if args.workload == "batch":
        return run_batch_workload(args)
    if args.workload == "precision":
        return run_precision_workload(args)
    if args.workload == "serving":
        return run_serving_workload(args)
    if args.workload == "edit":
        return run_edit_workload(args)
    if args.workload == "local":
        return run_local_workload(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

"""Benchmark: grid resistance (skyline + gres of every skyline tuple) on GB300.

One step = one gres_compute call over a resident synthetic dataset: the
sort-by-sum skyline pass, the candidate partitioning and the tile-pruned
grid-dominance kernel. Default workload: uniform N=1,000,000, d=6, values in
[0, 2^20), 256 log-spaced integer widths 1 .. 2^16, Angular partitioning (m=2,
32 partitions). The same line carries the Sliced (p=64) and no-partitioning
arms of that configuration and the anticorrelated N=100,000, d=4 configuration
(Grid m=4) as extra keys.

Metric: effective grid-dominance tests per second. Effective tests of one
step = S * sum_t min(k*(t) + 1, K): the (candidate, width) tests of the plain
early-exit scan of Algorithm 1 with the skyline as candidates (S candidates at
each width up to the exit width). It depends only on the result. The line
also gives executed_ops_per_s: the compare lane-ops the pruned kernel really
ran, per step time.

Prints one JSON line (rank 0). Timing: W warm-up steps; R repeats of exactly K
timed steps (R sized so that the repeats last about --clock-seconds, for the
clock sampler), each step bracketed by CUDA events on the launching stream,
with a 256 MiB write flushing L2 between steps (outside the events); barrier +
synchronize around each K steps; the median repeat, max over ranks. Under
torchrun each rank runs its own dataset instance (seed = rank) on its own GPU:
weak scaling, no collective on the data path.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2412_02274_gb300.inputs import make_dataset, steps_log, steps_linear  # noqa: E402

# workload name -> (distribution, n, d, value bits, steps, partition scheme, m, p)
WORKLOADS = {
    "ant-n100000-d4-b20-k256-grid-m4": ("ant", 100_000, 4, 20, ("log", 256, 16), "grid", 4, 0),
    "uni-n1000000-d6-b20-k256-angular-m2": ("uni", 1_000_000, 6, 20, ("log", 256, 16), "angular", 2, 0),
    "uni-n1000000-d6-b20-k256-sliced-p64": ("uni", 1_000_000, 6, 20, ("log", 256, 16), "sliced", 0, 64),
    "uni-n1000000-d6-b20-k256-none": ("uni", 1_000_000, 6, 20, ("log", 256, 16), "none", 0, 0),
    "uni-n1000-d2-b16-k64-grid": ("uni", 1_000, 2, 16, ("lin", 64, 64), "grid", 0, 0),
}
DEFAULT_WORKLOAD = "uni-n1000000-d6-b20-k256-angular-m2"
# arms printed in the same line as the workload: the same configuration with the other
# partitioning schemes, and the other single-GPU configuration
ARMS = {
    "uni-n1000000-d6-b20-k256-angular-m2": ("uni-n1000000-d6-b20-k256-sliced-p64", "uni-n1000000-d6-b20-k256-none",
                                            "ant-n100000-d4-b20-k256-grid-m4"),
}
MULTI_WORKLOADS = ("batch-512", "serve-10k", "sweep")
SCHEMES = {"none": 0, "grid": 1, "angular": 2, "sliced": 3}
METRIC = "effective grid-dominance tests/s (skyline + gres of every skyline tuple)"
UNIT = "tests/s"


def workload_inputs(name: str, seed: int):
    dist, n, d, bits, st, scheme, m, p = WORKLOADS[name]
    data = make_dataset(dist, n, d, bits=bits, seed=seed)
    steps = steps_log(st[1], st[2]) if st[0] == "log" else steps_linear(st[1], st[2])
    return data, steps, scheme, m, p


def effective_tests(step_idx: np.ndarray, K: int) -> int:
    S = len(step_idx)
    return int(S) * int(np.minimum(step_idx.astype(np.int64) + 1, K).sum())


# ---- clocks during the timed region --------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        time.sleep(0.3)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---- roofline bookkeeping ----------------------------------------------------------
def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def kernel_source_hash() -> str:
    src = os.path.join(ROOT, "paper_2412_02274_gb300", "csrc", "gres_stage.cu")
    with open(src, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def profiled_traffic(workload: str):
    """DRAM bytes per launch of the dominance kernel from a committed ncu summary,
    only if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", f"k_dominance_{workload}.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    h = re.search(r"source_sha256_16:\s*([0-9a-f]{16})", text)
    b = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not h or not b or h.group(1) != kernel_source_hash():
        return None
    return float(b.group(1))


# ---- the oracle on the host cores (baseline and reference arm) --------------------
def oracle_full(data, steps, threads: int):
    """The oracle on the whole workload, measured: BNL skyline of every row, then gres of
    every skyline tuple over the skyline as candidates (OpenMP over targets)."""
    from oracle import oracle as O
    t0 = time.perf_counter()
    sky = O.skyline_bnl(data)
    t_sky = time.perf_counter() - t0
    t0 = time.perf_counter()
    res = O.gres(data, steps, candidates=sky, targets=sky, threads=threads)
    t_gres = time.perf_counter() - t0
    eff = effective_tests(res, len(steps))
    secs = t_sky + t_gres
    return {"value": eff / secs if secs > 0 else 0.0, "seconds": secs, "skyline_s": t_sky,
            "gres_s": t_gres, "S": len(sky), "effective_tests": eff}


def run_reference(args):
    """The oracle as the reference arm. The skyline (BNL over every row) is computed and
    timed once before the warm-up. Step i then runs the oracle's gres for the skyline
    tuples j with j % Q == i % Q (a rotating, evenly spread slice; Q = --ref-slices), so
    that Q consecutive steps cover the whole workload once. Each step's time is its
    measured gres time plus Q-th of the measured skyline time; the value is the effective
    tests of the timed steps over their summed time."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import oracle as O
    threads = os.cpu_count() or 1
    data, steps, *_ = workload_inputs(args.workload, 0)
    K = len(steps)
    t0 = time.perf_counter()
    sky = O.skyline_bnl(data)
    skyline_s = time.perf_counter() - t0
    S = len(sky)
    Q = max(1, min(args.ref_slices, S)) if S else 1

    def step(i):
        tg = sky[(i % Q)::Q]
        t = time.perf_counter()
        r = O.gres(data, steps, candidates=sky, targets=tg, threads=threads)
        dt = time.perf_counter() - t + skyline_s / Q
        return dt, S * int(np.minimum(r.astype(np.int64) + 1, K).sum())

    for i in range(args.warmup):
        step(i)
    secs, units, per = 0.0, 0, []
    for i in range(args.steps):
        dt, u = step(i)
        secs += dt
        units += u
        per.append(dt)
    value = units / secs if secs > 0 else 0.0
    sample = (f"BNL skyline of all {len(data)} rows (measured once: {skyline_s:.2f} s, charged 1/{Q} per "
              f"step), then per step gres of every {Q}-th skyline tuple (rotating offset; S={S}) against "
              f"all S; {Q} consecutive steps cover the whole workload")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * secs / max(args.steps, 1), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": args.workload},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "step_s": {"min": min(per) if per else None, "median": statistics.median(per) if per else None,
                   "max": max(per) if per else None},
        "skyline_s": skyline_s,
    }
    print(json.dumps(line), flush=True)
    return 0


# ---- whole-job numbers over ranks ----------------------------------------------------
def _rank_reduce(x: float, op: str, device) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def rank_max(x: float, device) -> float:
    """The largest x over all ranks (x itself without a process group)."""
    return _rank_reduce(x, "max", device)


def rank_sum(x: float, device) -> float:
    """The sum of x over all ranks (x itself without a process group)."""
    return _rank_reduce(x, "sum", device)


def whole_job(total_ms: float, units: float, device):
    """(slowest rank's time, units of all ranks, units of all ranks / slowest time in s)."""
    t = rank_max(total_ms, device)
    u = rank_sum(units, device)
    return t, u, (u / (t / 1e3) if t > 0 else 0.0)


def repeats_for(target_s: float, est_repeat_ms: float, lo: int = 1, hi: int = 400) -> int:
    """Repeats of the K-step timed loop that keep the GPU busy for about target_s seconds
    (so the clock sampler sees the timed region), clamped to [lo, hi]."""
    if target_s <= 0 or est_repeat_ms <= 0:
        return lo
    return int(max(lo, min(hi, round(target_s * 1e3 / est_repeat_ms))))


def measure_test_peak(G, torch, d: int, dev, stream, iters: int = 4096, reps: int = 5) -> dict:
    """Measured peak of the dominance test on this GPU: the library's probe kernel (every
    thread tests 16 register-held candidates per iteration, 2d compare lane-ops each), one
    full wave of blocks, timed with CUDA events on `stream`; median of `reps` launches.
    The bench probes at d = 4 whatever the workload's d: that pattern keeps the ALU pipe 98%
    busy (ncu). The same probe at d = 6 (127 registers, 16 warps per SM instead of 24) measured 6.7 T
    lane-ops/s, a limit of the probe's code, not of the pipe."""
    sink = torch.zeros(1, dtype=torch.int64, device=dev)
    G.test_peak_probe(d, iters, sink, stream=stream)
    rates = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ops = G.test_peak_probe(d, iters, sink, stream=stream)
        b.record(stream)
        b.synchronize()
        rates.append(ops / (a.elapsed_time(b) / 1e3))
    return {"lane_ops_per_s": float(statistics.median(rates)), "d": d, "iters": iters, "launches": reps}


def alu_peak(torch, dev, clocks) -> tuple[float, str]:
    """The ALU-pipe peak in lane-ops/s: integer compare / logic / min-max issue to the ALU
    pipe, 16 lanes per clock per SM sub-partition, 64 per SM, at the maximum SM clock."""
    props = torch.cuda.get_device_properties(dev)
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz") or clocks.get("sm_max_mhz") or 2070.0)
    lanes = 64
    return (props.multi_processor_count * lanes * sm_max * 1e6,
            f"{props.multi_processor_count} SMs x {lanes} ALU-pipe lanes x {sm_max:.0f} MHz (max SM clock)")


# ---- our arm ------------------------------------------------------------------------
class Arm:
    """One workload on the device: the dataset resident in HBM, a workspace, one CUDA graph
    of one gres_compute per timed step (or direct calls), the result of the warm-up and the
    counters of a separate counted run."""

    def __init__(self, G, torch, name, seed, dev, stream, steps, warmup, graph):
        self.G, self.torch, self.name, self.dev, self.stream = G, torch, name, dev, stream
        self.data, self.widths, self.scheme, self.m, self.p = workload_inputs(name, seed)
        self.n, self.d = self.data.shape
        self.K = len(self.widths)
        self.cfg = G.plan(SCHEMES[self.scheme], m=self.m, p=self.p)
        self.x = G.to_device_u32(self.data, dev)
        self.ws = G.alloc_workspace(self.n, self.d, self.K)
        self.out = (torch.empty(self.n, dtype=torch.int64, device=dev),
                    torch.empty(self.n, dtype=torch.int32, device=dev),
                    torch.zeros(1, dtype=torch.int64, device=dev))
        for _ in range(warmup):
            self.call(stream)
        torch.cuda.synchronize(dev)
        self.S = int(self.out[2].item())
        self.step_idx = self.out[1][:self.S].cpu().numpy()
        self.sky_idx = self.out[0][:self.S].cpu().numpy()
        self.eff = effective_tests(self.step_idx, self.K)
        # executed (candidate, width) lane-tests and pruning checks of the dominance kernel
        tests = torch.zeros(2, dtype=torch.int64, device=dev)
        cfg_c = G.plan(SCHEMES[self.scheme], m=self.m, p=self.p, count_tests=True)
        G.gres_compute(self.x, self.widths, G.MIN, cfg_c, ws=self.ws, sync=False, out=self.out, stream=stream,
                       tests=tests)
        torch.cuda.synchronize(dev)
        self.executed, self.checks = (int(v) for v in tests.cpu().tolist())
        # stage events: each timed step replays its own captured graph, whose event record
        # nodes give that step's stage durations (stage_times reads the last replay of
        # each graph); timing stays on until then
        G.timing_enable(True)
        self.graphs = []
        self.launches_per_call = None
        if graph:
            cap = torch.cuda.Stream(dev)
            cap.wait_stream(stream)
            for _ in range(steps):
                g = torch.cuda.CUDAGraph()
                c0 = G.launch_count()
                with torch.cuda.graph(g, stream=cap):
                    self.call(cap)
                self.launches_per_call = G.launch_count() - c0
                self.graphs.append(g)
            torch.cuda.synchronize(dev)
            for i in range(warmup):
                self.graphs[i % len(self.graphs)].replay()
            torch.cuda.synchronize(dev)
        else:
            G.timing_enable(False)

    def call(self, stream):
        self.G.gres_compute(self.x, self.widths, self.G.MIN, self.cfg, ws=self.ws, sync=False, out=self.out,
                            stream=stream)

    def timed_loop(self, steps, flush, world):
        """Exactly `steps` steps, each bracketed by CUDA events on the launching stream, with
        an L2 flush (a 256 MiB write) before each, outside the events; barrier +
        synchronize on both sides. Returns (per-step ms, kernels launched)."""
        import torch.distributed as dist
        torch, G, stream, dev = self.torch, self.G, self.stream, self.dev
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        c0 = G.launch_count()
        for i in range(steps):
            flush.zero_()
            starts[i].record(stream)
            if self.graphs:
                self.graphs[i].replay()
            else:
                self.call(stream)
            ends[i].record(stream)
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        launches = (self.launches_per_call * steps) if self.graphs else G.launch_count() - c0
        return [s.elapsed_time(e) for s, e in zip(starts, ends)], launches

    def check_result(self):
        """The timed steps give the warm-up's result."""
        assert int(self.out[2].item()) == self.S
        assert np.array_equal(self.out[1][:self.S].cpu().numpy(), self.step_idx)

    def stage_times(self, steps, flush, world):
        """Per-stage (total ms, launches) of one timed loop, from the library's stage events:
        with graphs, those of the last replay of each graph (the loop just run); with direct
        calls, one more loop with timing on."""
        G = self.G
        if not self.graphs:
            G.timing_enable(True)
            self.timed_loop(steps, flush, world)
        st = G.timing_read()
        G.timing_enable(False)
        return st

    def summary(self, step_ms_mean, stages, peak_ops):
        """The arm's numbers for the JSON line."""
        dom_ms, dom_n = stages.get("dominance", (0.0, 0))
        dom_avg_s = (dom_ms / dom_n) / 1e3 if dom_n else None
        alg_ops = (self.executed + self.checks) * 2 * self.d
        achieved = alg_ops / dom_avg_s if dom_avg_s else 0.0
        return {"workload": self.name, "n": int(self.n), "d": int(self.d), "widths": self.K,
                "scheme": self.scheme, "m": self.m, "p": self.p, "skyline_size": self.S,
                "ms_per_step": step_ms_mean, "value": self.eff / (step_ms_mean / 1e3) if step_ms_mean else None,
                "unit": UNIT, "effective_tests_per_step": self.eff,
                "executed_lane_tests_per_step": self.executed, "pruning_checks_per_step": self.checks,
                "executed_ops_per_s": alg_ops / (step_ms_mean / 1e3) if step_ms_mean else None,
                "stage_ms_per_step": {k: (v[0] / v[1] if v[1] else None) for k, v in stages.items()},
                "dominance": {"ops_per_launch": alg_ops, "avg_launch_ms": dom_avg_s * 1e3 if dom_avg_s else None,
                              "achieved_tops": achieved / 1e12, "frac_of_alu_peak": achieved / peak_ops}}

    def close(self):
        self.graphs = []
        self.x = self.ws = self.out = None


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2412_02274_gb300 import gres as G

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group(backend="nccl")
    dev = torch.device("cuda", local if world > 1 else torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)

    arm = Arm(G, torch, args.workload, rank, dev, stream, args.steps, args.warmup, args.graph)
    n, d, K, S = arm.n, arm.d, arm.K, arm.S

    # Timed region: R repeats of exactly K steps (R sized so that the repeats keep the GPU
    # busy for about --clock-seconds, long enough for the clock sampler to see them); the
    # reported time is the median repeat.
    probe_ms, _ = arm.timed_loop(args.steps, flush, world)
    R = repeats_for(args.clock_seconds, float(sum(probe_ms)) * 1.3)
    R = int(rank_max(R, dev))
    sampler = ClockSampler(dev.index if dev.index is not None else 0)
    sampler.start()
    rep_ms, launches = [], 0
    for _ in range(R):
        ms, l = arm.timed_loop(args.steps, flush, world)
        rep_ms.append(float(sum(ms)))
        launches = l
    clocks = sampler.stop()
    arm.check_result()
    med_ms = float(statistics.median(rep_ms))
    total_ms, total_eff, value = whole_job(med_ms, float(arm.eff) * args.steps, dev)
    ms_per_step = total_ms / args.steps

    # stage durations of the dominant kernel (the grid-dominance kernel) and the others
    stages = arm.stage_times(args.steps, flush, world)
    peak_ops, peak_basis = alu_peak(torch, dev, clocks)
    main = arm.summary(ms_per_step, stages, peak_ops)
    dom = main["dominance"]
    traffic = profiled_traffic(args.workload)
    probe = measure_test_peak(G, torch, 4, dev, stream)
    achieved = dom["achieved_tops"] * 1e12
    roofline = {"bound": "alu", "achieved": dom["achieved_tops"], "peak": peak_ops / 1e12,
                "unit": "Tops/s", "frac": achieved / peak_ops if peak_ops else None,
                "traffic": traffic, "kernel": "k_dominance", "peak_basis": peak_basis,
                "peak_measured": probe["lane_ops_per_s"] / 1e12,
                "frac_of_measured": achieved / probe["lane_ops_per_s"] if probe["lane_ops_per_s"] else None,
                "peak_measured_basis": f"dominance-test probe (gres_test_peak_probe), d={probe['d']}, "
                f"16 register-held candidates per thread, one wave, median of {probe['launches']} launches",
                "ops_per_launch": dom["ops_per_launch"], "avg_launch_ms": dom["avg_launch_ms"],
                "ops_basis": "(executed lane-tests + pruning checks) x 2d unsigned compares, from a counted run"}

    # end to end through the host-buffer ABI: pinned input, H2D + compute + D2H each step
    pinned = torch.from_numpy(arm.data.view(np.int32)).pin_memory()
    ws_h = G.alloc_workspace(n, d, K, host=True)
    hs = torch.empty(n, dtype=torch.int64).pin_memory()
    hr = torch.empty(n, dtype=torch.int32).pin_memory()
    for _ in range(max(1, args.warmup)):
        G.gres_compute_host(pinned, arm.widths, G.MIN, arm.cfg, ws=ws_h, out=(hs, hr), stream=stream)
    torch.cuda.synchronize(dev)
    # each call returns after its results are on the host, so host wall-clock time around it is
    # the call's end-to-end time; the L2 flush before each call stays outside the timed part
    e2e_total = 0.0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        sk, rr = G.gres_compute_host(pinned, arm.widths, G.MIN, arm.cfg, ws=ws_h, out=(hs, hr), stream=stream)
        e2e_total += time.perf_counter() - t0
    e2e_s = e2e_total / args.steps
    assert np.array_equal(rr.numpy(), arm.step_idx)
    e2e_s_all = rank_max(e2e_s, dev)
    e2e = {"value": total_eff / args.steps / e2e_s_all, "unit": UNIT,
           "h2d_bytes_per_step": int(n * d * 4), "d2h_bytes_per_step": int(S * 12 + 8),
           "ms_per_step": e2e_s_all * 1e3}
    del ws_h, pinned

    # the other arms of the same configuration and the other single-GPU configuration, on
    # rank 0 (each with its own warm-up and K graph-replayed steps)
    others = {}
    if rank == 0 and not args.no_arms:
        for name in ARMS.get(args.workload, ()):
            a = Arm(G, torch, name, rank, dev, stream, args.steps, args.warmup, args.graph)
            ms, _ = a.timed_loop(args.steps, flush, 1)
            st = a.stage_times(args.steps, flush, 1)
            a.check_result()
            if a.data.shape == arm.data.shape and np.array_equal(a.data, arm.data) and \
                    (a.S != S or not np.array_equal(a.step_idx, arm.step_idx)):
                raise RuntimeError(f"{name}: results differ from {args.workload}")
            others[name] = a.summary(float(sum(ms)) / args.steps, st, peak_ops)
            a.close()
            torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        r = oracle_full(arm.data, arm.widths, threads)
        if r["S"] != S:
            raise RuntimeError("oracle skyline size differs from the GPU's")
        cpu = {"value": r["value"], "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"the whole workload, measured: BNL skyline of all {n} rows ({r['skyline_s']:.2f} s) "
                         f"+ gres of all S={r['S']} skyline tuples against all S ({r['gres_s']:.2f} s, "
                         f"OpenMP over targets); {r['seconds']:.1f} s of CPU wall time",
               "seconds": r["seconds"]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": args.workload, "n": int(n), "d": int(d), "value_bits": WORKLOADS[args.workload][3],
                       "widths": K, "scheme": arm.scheme, "m": arm.m, "p": arm.p, "skyline_size": S,
                       "effective_tests_per_step": arm.eff, "executed_lane_tests_per_step": arm.executed,
                       "pruning_checks_per_step": arm.checks,
                       "l2": "256 MiB write between timed steps (device-timed and end-to-end)",
                       "seed_per_rank": "rank",
                       "launch": "cuda graph replay" if args.graph else "direct calls",
                       "timed_region": f"{R} repeats of exactly {args.steps} steps; the median repeat is reported",
                       "parallelism": f"replicas x{world} (one dataset per GPU)"},
            "executed_ops_per_s": main["executed_ops_per_s"],
            "effective_vs_executed": "value counts the tests of the plain early-exit scan (S candidates at "
                                     "every width up to each exit); executed_ops_per_s counts the compare "
                                     "lane-ops the pruned kernel actually ran, per step time",
            "gres_queries_per_s": world * 1e3 / ms_per_step,
            "stage_ms_per_step": main["stage_ms_per_step"],
            "repeats": {"count": R, "ms_min": min(rep_ms), "ms_median": med_ms, "ms_max": max(rep_ms)},
            "roofline": roofline,
            "arms": others,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "launches_per_step": int(launches // max(args.steps, 1)),
            "clocks": clocks,
        }
        if clocks.get("sm_mhz"):
            line["cycles_per_step"] = ms_per_step * 1e-3 * clocks["sm_mhz"] * 1e6
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


# ---- many instances (one gres_batch per step) ------------------------------------
def batch_problems(count=512, seed=0):
    """512 instances: N log-uniform in [1e3, 2e5], d in {2..8}, UNI / ANT (0.05) /
    CLU (16 clusters, 0.02), values in [0, 2^20), 128 log-spaced widths."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(round(np.exp(rng.uniform(np.log(1e3), np.log(2e5)))))
        d = int(rng.integers(2, 9))
        dist = ("uni", "ant", "clu")[int(rng.integers(0, 3))]
        out.append((dist, n, d, make_dataset(dist, n, d, bits=20, seed=seed * 100000 + i)))
    return out, steps_log(128, 16)


def _time_batch(probs, args, dev, stream):
    """One gres_batch over probs captured in a CUDA graph; mean replay ms, launches per call,
    clocks and the outputs."""
    import torch
    from paper_2412_02274_gb300 import gres as G
    outs, cinsts, ws = G.batch(probs, stream=stream)
    torch.cuda.synchronize(dev)
    lib = G.load()
    graph = torch.cuda.CUDAGraph()
    cap = torch.cuda.Stream(dev)
    cap.wait_stream(stream)
    c0 = G.launch_count()
    with torch.cuda.graph(graph, stream=cap):
        G._check(lib.gres_batch(cinsts, len(probs), G._ptr(ws), ws.numel(), G._stream_ptr(cap)))
    per_call = G.launch_count() - c0
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)
    sampler = ClockSampler(dev.index or 0)
    sampler.start()
    t_ms = []
    for _ in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        graph.replay()
        b.record(stream)
        torch.cuda.synchronize(dev)
        t_ms.append(a.elapsed_time(b))
    clocks = sampler.stop()
    del graph
    return float(np.mean(t_ms)), per_call, clocks, outs


def run_batch(args):
    import torch
    from paper_2412_02274_gb300 import gres as G
    from paper_2412_02274_gb300.autotune import Autotuner
    dev = torch.device("cuda", torch.cuda.current_device())
    insts, steps = batch_problems()
    K = len(steps)
    tsteps = torch.from_numpy(steps.view(np.int32)).to(dev)
    datas = [G.to_device_u32(data, dev) for _, _, _, data in insts]
    stream = torch.cuda.current_stream(dev)
    # default plan (Grid, about 256 cells, 8 slots) for every instance
    dflt = [{"data": x, "steps": tsteps, "cfg": G.plan(G.PART_GRID)} for x in datas]
    ms_default, _, _, outs_d = _time_batch(dflt, args, dev, stream)
    # autotuned plans: candidates timed per size class (d, power-of-two bucket of n) on
    # the two largest instances of the class, outside the timed region, scored as part
    # of a batch (the dominance stage plus the overlapped other stages / 16)
    t0 = time.time()
    tuner = Autotuner(objective="batch")
    table = tuner.tune(datas, steps, samples_per_class=2)
    tune_s = time.time() - t0
    probs = [{"data": x, "steps": tsteps, "cfg": tuner.plan_for(int(x.shape[0]), int(x.shape[1]))}
             for x in datas]
    ms, per_call, clocks, outs = _time_batch(probs, args, dev, stream)
    eff = 0
    for (sky, res, cnt), (sky_d, res_d, cnt_d) in zip(outs, outs_d):
        S = int(cnt.item())
        r = res[:S].cpu().numpy()
        if S != int(cnt_d.item()) or not np.array_equal(r, res_d[:S].cpu().numpy()):
            raise RuntimeError("tuned and default plans disagree")
        eff += effective_tests(r, K)
    # the same 512 problems one at a time (one gres_compute per instance, direct calls)
    wss = {}
    for _ in range(max(1, args.warmup // 2)):
        for pr in probs:
            n, d = pr["data"].shape
            key = (int(n), int(d))
            if key not in wss:
                wss[key] = G.alloc_workspace(int(n), int(d), K)
            G.gres_compute(pr["data"], steps, G.MIN, pr["cfg"], ws=wss[key], sync=False, stream=stream)
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for pr in probs:
        n, d = pr["data"].shape
        G.gres_compute(pr["data"], steps, G.MIN, pr["cfg"], ws=wss[(int(n), int(d))], sync=False,
                       stream=stream)
    b.record(stream)
    torch.cuda.synchronize(dev)
    ms_single = a.elapsed_time(b)
    # the same single calls captured into one CUDA graph (one stream, in order), replayed:
    # one at a time without the host's launch overhead
    cap = torch.cuda.Stream(dev)
    cap.wait_stream(stream)
    g1 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g1, stream=cap):
        for pr in probs:
            n, d = pr["data"].shape
            G.gres_compute(pr["data"], steps, G.MIN, pr["cfg"], ws=wss[(int(n), int(d))], sync=False, stream=cap)
    for _ in range(2):
        g1.replay()
    torch.cuda.synchronize(dev)
    t_g = []
    l2flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)
    for _ in range(max(3, args.steps // 2)):
        l2flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        g1.replay()
        b.record(stream)
        torch.cuda.synchronize(dev)
        t_g.append(a.elapsed_time(b))
    ms_single_graph = float(np.median(t_g))
    del g1
    picks = {}
    for name in table.values():
        picks[name] = picks.get(name, 0) + 1
    line = {"metric": "gres instances/s (512 uneven instances per step)", "value": len(probs) / (ms / 1e3),
            "unit": "instances/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic",
            "config": {"workload": "batch-512", "instances": len(probs), "widths": K,
                       "n_range": [1000, 200000], "d_range": [2, 8], "distributions": ["uni", "ant", "clu"],
                       "launch": "one gres_batch captured in a CUDA graph", "plans": "autotuned",
                       "l2": "256 MiB write between timed steps"},
            "effective_tests_per_s": eff / (ms / 1e3),
            "default_plan": {"ms": ms_default, "instances_per_s": len(probs) / (ms_default / 1e3)},
            "autotune": {"classes": len(table), "seconds": tune_s, "picks": picks},
            "one_at_a_time": {"ms": ms_single, "instances_per_s": len(probs) / (ms_single / 1e3),
                              "speedup_of_batch": ms_single / ms},
            "one_at_a_time_graph": {"ms": ms_single_graph,
                                    "instances_per_s": len(probs) / (ms_single_graph / 1e3),
                                    "speedup_of_batch": ms_single_graph / ms,
                                    "launch": "the 512 single calls captured in one CUDA graph on one stream"},
            "gpu_launches": per_call * args.steps, "clocks": clocks}
    if args.tune_table:
        with open(args.tune_table, "w") as f:
            f.write(tuner.to_json())
    print(json.dumps(line), flush=True)
    return 0


# ---- the paper's operating-parameter sweep (Table 1) ---------------------------------
def table1_plan(scheme: str, d: int, p_target: int):
    """(m or p) closest to the target partition count, with more than one partition (as the
    paper does for Grid m^d and Angular m^(d-1))."""
    if scheme in ("grid", "angular"):
        dims = d if scheme == "grid" else d - 1
        if dims < 1:
            return 1, 1
        best = None
        for m in range(2, 65):
            cells = m ** dims
            if cells >= 1 << 32:
                break
            score = abs(np.log(cells) - np.log(p_target))
            if best is None or score < best[0]:
                best = (score, m, cells)
        return best[1], best[2]
    if scheme == "sliced":
        return p_target, p_target
    return 0, 1


def run_sweep(args):
    """Dominance tests and time per partitioning scheme over the paper's operating
    parameters (Table 1): N, d, partitions, representatives; UNI and ANT; the practical
    g_bar = 25 (g = 25 .. 2) on 20-bit values. Counters: lane-tests of the grid-dominance
    kernel and pruning checks (GRES_FLAG_COUNT_TESTS)."""
    import torch
    from paper_2412_02274_gb300 import gres as G
    dev = torch.device("cuda", torch.cuda.current_device())
    glist = np.arange(25, 1, -1, dtype=np.uint32)
    configs = []
    for dist in ("uni", "ant"):
        for n in (100_000, 500_000, 1_000_000, 5_000_000, 10_000_000):
            configs.append((dist, n, 3, 16, 0))
        for d in (2, 4, 5, 6, 7):
            configs.append((dist, 1_000_000, d, 16, 0))
        for p in (32, 64, 128):
            configs.append((dist, 1_000_000, 3, p, 0))
        for reps in (1, 10, 100, 1000):
            configs.append((dist, 1_000_000, 3, 16, reps))
    rows = []
    stream = torch.cuda.current_stream(dev)
    for dist, n, d, p_target, reps in configs:
        data = make_dataset(dist, n, d, bits=20, seed=0)
        x = G.to_device_u32(data, dev)
        ws = G.alloc_workspace(n, d, len(glist))
        for scheme in ("grid", "angular", "sliced", "none"):
            mp, cells = table1_plan(scheme, d, p_target)
            kw = {"m": mp} if scheme in ("grid", "angular") else ({"p": mp} if scheme == "sliced" else {})
            cfg = G.plan(SCHEMES[scheme], reps=reps, **kw)
            G.gres_compute_g(x, 20, glist, G.MIN, cfg, ws=ws, stream=stream)    # warm-up
            # counters split by partition (GRES_FLAG_COUNT_PARTS): the paper's phases
            cfg_c = G.plan(SCHEMES[scheme], reps=reps, count_parts=True, **kw)
            P = G.plan_partitions(cfg_c, d)
            tests = torch.zeros(2 + 4 * P, dtype=torch.int64, device=dev)
            sky, idx = G.gres_compute_g(x, 20, glist, G.MIN, cfg_c, ws=ws, stream=stream, tests=tests)
            tv = tests.cpu().numpy()
            lane_tests, checks = int(tv[0]), int(tv[1])
            split = tv[2:].reshape(P, 4)
            G.timing_enable(True)
            G.timing_read()
            t = []
            for _ in range(3):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                G.gres_compute_g(x, 20, glist, G.MIN, cfg, ws=ws, stream=stream)
                b.record(stream)
                b.synchronize()
                t.append(a.elapsed_time(b))
            st = G.timing_read()
            G.timing_enable(False)
            S = int(sky.numel())
            rows.append({"dist": dist, "n": n, "d": d, "p_target": p_target, "reps": reps or 1024,
                         "scheme": scheme, "param": mp, "partitions": cells, "S": S,
                         "lane_tests": lane_tests, "pruning_checks": checks,
                         # the paper's accounting: parallel phase = the heaviest partition's work
                         # against its own candidates, final phase = all work across partitions
                         "parallel_phase_lane_tests": int(split[:, 0].max()),
                         "final_phase_lane_tests": int(split[:, 2].sum()),
                         "parallel_phase_row_checks": int(split[:, 1].max()),
                         "final_phase_row_checks": int(split[:, 3].sum()),
                         "local_lane_tests": int(split[:, 0].sum()),
                         "dense_tests": S * S * len(glist),
                         "ms": float(np.median(t)), "skyline_ms": st["skyline"][0] / max(st["skyline"][1], 1),
                         "partition_ms": st["partition"][0] / max(st["partition"][1], 1),
                         "dominance_ms": st["dominance"][0] / max(st["dominance"][1], 1)})
            print(json.dumps({"row": rows[-1]}), file=sys.stderr, flush=True)
        del x, ws
        torch.cuda.empty_cache()
    # Representative Filtering inside the gres stage (32 representatives), against the plain search
    ablation = []
    for dist, n, d in (("ant", 1_000_000, 3), ("ant", 1_000_000, 5), ("uni", 1_000_000, 6),
                       ("ant", 100_000, 4)):
        data = make_dataset(dist, n, d, bits=20, seed=0)
        x = G.to_device_u32(data, dev)
        ws = G.alloc_workspace(n, d, len(glist))
        for scheme in ("grid", "sliced"):
            mp, cells = table1_plan(scheme, d, 16)
            kw = {"m": mp} if scheme == "grid" else {"p": mp}
            for reps_on in (False, True):
                cfg = G.plan(SCHEMES[scheme], gres_reps=reps_on, **kw)
                G.gres_compute_g(x, 20, glist, G.MIN, cfg, ws=ws, stream=stream)
                tests = torch.zeros(2, dtype=torch.int64, device=dev)
                G.gres_compute_g(x, 20, glist, G.MIN, G.plan(SCHEMES[scheme], gres_reps=reps_on, count_tests=True, **kw),
                                 ws=ws, stream=stream, tests=tests)
                lane_tests, checks = (int(v) for v in tests.cpu().tolist())
                G.timing_enable(True)
                G.timing_read()
                t = []
                for _ in range(3):
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    G.gres_compute_g(x, 20, glist, G.MIN, cfg, ws=ws, stream=stream)
                    b.record(stream)
                    b.synchronize()
                    t.append(a.elapsed_time(b))
                st = G.timing_read()
                G.timing_enable(False)
                ablation.append({"dist": dist, "n": n, "d": d, "scheme": scheme, "gres_reps": 32 if reps_on else 0,
                                 "lane_tests": lane_tests, "pruning_checks": checks, "ms": float(np.median(t)),
                                 "dominance_ms": st["dominance"][0] / max(st["dominance"][1], 1)})
                print(json.dumps({"ablation": ablation[-1]}), file=sys.stderr, flush=True)
        del x, ws
        torch.cuda.empty_cache()
    line = {"metric": "dominance tests and time per scheme (Table 1 sweep)", "value": len(rows),
            "unit": "configurations", "n_gpus": 1, "steps": 3, "warmup": 1, "ms_per_step": None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": {"workload": "sweep", "g": "25..2", "value_bits": 20,
                                            "seed": 0}, "rows": rows, "gres_reps_ablation": ablation}
    print(json.dumps(line), flush=True)
    return 0


# ---- serving ----------------------------------------------------------------------
def serve_datasets(count=64, seed=1):
    """64 datasets: N log-uniform in [1e3, 2e6], d in {2..8}, UNI / ANT / CLU mix."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(round(np.exp(rng.uniform(np.log(1e3), np.log(2e6)))))
        d = int(rng.integers(2, 9))
        dist = ("uni", "ant", "clu")[i % 3]
        out.append(make_dataset(dist, n, d, bits=20, seed=seed * 100000 + i))
    return out


def run_serve(args):
    import torch
    from paper_2412_02274_gb300 import gres as G
    rng = np.random.default_rng(2)
    datas = serve_datasets()
    sv = G.Server(64 << 30, max_batch=128, max_inflight=3, chunk_targets=args.chunk_targets)
    ids = [sv.add_dataset(x, G.MIN, G.plan(G.PART_GRID)) for x in datas]
    nq = 10000
    qs = [(ids[int(rng.integers(0, len(ids)))], steps_log(int(rng.integers(64, 257)), 16)) for _ in range(nq)]
    # warm-up
    for t in [sv.submit(i, st) for i, st in qs[:200]]:
        sv.poll(t)
    # saturation: every query at once
    t0 = time.perf_counter()
    tickets = [sv.submit(i, st) for i, st in qs]
    lats = [sv.poll(t)[1] for t in tickets]
    sat_s = time.perf_counter() - t0
    sat_qps = nq / sat_s
    # Poisson arrivals at 80 % of the saturating rate
    lam = 0.8 * sat_qps
    gaps = rng.exponential(1.0 / lam, size=nq)
    done = []

    def poller(ts):
        for t in ts:
            done.append(sv.poll(t)[1])

    tickets = []
    t0 = time.perf_counter()
    nxt = t0
    for (i, st), g in zip(qs, gaps):
        nxt += g
        while time.perf_counter() < nxt:
            pass
        tickets.append(sv.submit(i, st))
    for t in tickets:
        done.append(sv.poll(t)[1])
    load_s = time.perf_counter() - t0
    lat = np.array(done) / 1e6
    stats = sv.stats()
    # one query at a time: each query alone, waiting for it before the next
    alone = [G.Dataset(x, G.MIN, G.plan(G.PART_GRID)) for x in datas]
    stream = torch.cuda.current_stream()
    qws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    outb = torch.empty(1 << 21, dtype=torch.int32, device="cuda")
    for i, st in qs[:100]:
        alone[i].query(st, out=outb, qws=qws, stream=stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    single = []
    for i, st in qs:        # the same 10,000 queries, each waited for before the next
        a = time.perf_counter()
        r = alone[i].query(st, out=outb, qws=qws, stream=stream)
        r.cpu()
        single.append(time.perf_counter() - a)
    single_qps = nq / (time.perf_counter() - t0)
    # one at a time under the same Poisson arrivals: a single worker serves the queries in
    # arrival order, each alone and waited for; latency = completion - arrival
    single_lat = []
    t0 = time.perf_counter()
    arrival = t0
    for (i, st), g in zip(qs, gaps):
        arrival += g
        while time.perf_counter() < arrival:
            pass
        r = alone[i].query(st, out=outb, qws=qws, stream=stream)
        r.cpu()
        single_lat.append(time.perf_counter() - arrival)
    single_load_s = time.perf_counter() - t0
    sv.close()
    line = {"metric": "gres queries/s served (10,000 queries on 64 resident datasets)", "value": sat_qps,
            "unit": "queries/s", "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": sat_s * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": {"workload": "serve-10k", "datasets": len(datas), "n_range": [1000, 2000000],
                       "d_range": [2, 8], "widths": [64, 256], "max_batch": 128, "max_inflight": 3,
                       "chunk_targets": args.chunk_targets or 16384},
            "saturation": {"qps": sat_qps, "p50_ms": float(np.percentile(lats, 50)) / 1e6,
                           "p99_ms": float(np.percentile(lats, 99)) / 1e6},
            "poisson_80pct": {"lambda_qps": lam, "achieved_qps": nq / load_s,
                              "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99))},
            "one_at_a_time": {"qps": single_qps, "service_p50_ms": 1e3 * float(np.percentile(single, 50)),
                              "service_p99_ms": 1e3 * float(np.percentile(single, 99)),
                              "poisson_80pct": {"lambda_qps": lam, "achieved_qps": nq / single_load_s,
                                                "p50_ms": 1e3 * float(np.percentile(single_lat, 50)),
                                                "p99_ms": 1e3 * float(np.percentile(single_lat, 99))}},
            "server": stats}
    print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + list(MULTI_WORKLOADS), default=DEFAULT_WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--graph", action=argparse.BooleanOptionalAction, default=True,
                    help="each step replays a gres_compute captured in a CUDA graph "
                         "(--no-graph: direct calls)")
    ap.add_argument("--no-arms", action="store_true", help="leave out the extra arms of the line")
    ap.add_argument("--clock-seconds", type=float, default=2.0,
                    help="repeat the K timed steps for about this long (the median repeat is reported)")
    ap.add_argument("--ref-slices", type=int, default=4,
                    help="reference arm: each step runs the oracle's gres for every Q-th skyline tuple")
    ap.add_argument("--tune-table", default="", help="batch-512: write the autotuned plan table (JSON) here")
    ap.add_argument("--chunk-targets", type=int, default=0,
                    help="serve-10k: targets per query piece (0: the library default)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch-512":
        return run_batch(args)
    if args.workload == "serve-10k":
        return run_serve(args)
    if args.workload == "sweep":
        return run_sweep(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

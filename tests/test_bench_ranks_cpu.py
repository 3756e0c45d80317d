"""bench.py's multi-rank host logic on CPU: two gloo ranks (world size 2).

Each rank times its own replica (its own seed); the whole-job value is the
units of all ranks over the slowest rank's time, and only rank 0 prints.
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dev = torch.device("cpu")
    # rank r: 10 + 5 r ms for 100 (r + 1) units
    t, u, v = bench.whole_job(10.0 + 5.0 * rank, 100.0 * (rank + 1), dev)
    e2e = bench.rank_max(0.001 * (rank + 1), dev)
    data, steps, *_ = bench.workload_inputs("uni-n1000-d2-b16-k64-grid", seed=rank)
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"t": t, "u": u, "v": v, "e2e": e2e, "digest": int(data.astype(np.uint64).sum()),
                   "k": len(steps)}, f)


def test_whole_job_reduction_two_gloo_ranks(tmp_path):
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    r0 = json.load(open(tmp_path / "r0.json"))
    r1 = json.load(open(tmp_path / "r1.json"))
    for r in (r0, r1):
        assert r["t"] == 15.0 and r["u"] == 300.0
        assert abs(r["v"] - 300.0 / 0.015) < 1e-6
        assert r["e2e"] == 0.002
        assert r["k"] == 64
    assert r0["digest"] != r1["digest"]      # each rank works on its own replica (seed = rank)


def test_single_process_reduction_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job(20.0, 50.0, "cpu") == (20.0, 50.0, 2500.0)
    assert bench.rank_sum(3.0, "cpu") == 3.0


def test_reference_arm_prints_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                          "--steps", "1", "--warmup", "3"], env=env, capture_output=True, text=True,
                         timeout=300, cwd=ROOT)
    assert out.returncode == 0 and out.stdout.strip() == ""


def test_reference_arm_line_on_rank_zero():
    """The reference arm (the oracle on the host cores) runs without a GPU and prints one JSON
    line with the contract's keys; a small workload keeps it quick."""
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "uni-n1000-d2-b16-k64-grid", "--steps", "2", "--warmup", "3"],
                         env=env, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == "uni-n1000-d2-b16-k64-grid"

"""GPU: resident-dataset queries and multi-instance batches, bit-exact.

Each result is checked against the single-call path (gres_compute, itself
pinned to the oracle) and, for a subset, against the oracle directly.
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2412_02274_gb300 import gres as G
from paper_2412_02274_gb300.inputs import make_dataset, steps_log, steps_linear

pytestmark = pytest.mark.gpu

THREADS = max(1, os.cpu_count() or 1)


def _compute(data, steps, direction=G.MIN, cfg=None):
    sky, res = G.gres_compute(G.to_device_u32(data), steps, direction, cfg)
    return sky.cpu().numpy(), res.cpu().numpy()


def test_dataset_queries_match_single_calls():
    import torch
    data = make_dataset("ant", 30000, 4, bits=20, seed=11)
    for direction in (G.MIN, G.MAX):
        ds = G.Dataset(G.to_device_u32(data), direction, G.plan(G.PART_GRID, m=4))
        sky = ds.sky_idx()
        for steps in (steps_log(256, 16), steps_log(64, 12), steps_linear(40, 300),
                      np.arange(1, 700, dtype=np.uint32) * 13):
            ref_sky, ref_res = _compute(data, steps, direction, G.plan(G.PART_GRID, m=4))
            np.testing.assert_array_equal(sky, ref_sky)
            np.testing.assert_array_equal(ds.query(steps).cpu().numpy(), ref_res)
        ds.close()
    # from host memory, oracle directly
    data = make_dataset("clu", 8000, 3, bits=16, seed=2)
    ds = G.Dataset(data, G.MIN, G.plan(G.PART_SLICED, p=16))
    steps = steps_log(100, 14)
    osky = O.skyline_bnl(data)
    np.testing.assert_array_equal(ds.sky_idx(), osky)
    exp = O.gres(data, steps, candidates=osky, targets=osky, threads=THREADS)
    np.testing.assert_array_equal(ds.query(steps).cpu().numpy(), exp)
    # queries on two streams at once, each with its own scratch
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    a = ds.query(steps, stream=s1)
    b = ds.query(steps_log(30, 14), stream=s2)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(a.cpu().numpy(), exp)
    np.testing.assert_array_equal(b.cpu().numpy(), _compute(data, steps_log(30, 14))[1])
    ds.close()
    # an empty dataset
    ds = G.Dataset(np.zeros((0, 2), np.uint32))
    assert ds.S == 0 and len(ds.sky_idx()) == 0 and len(ds.query([1, 2])) == 0
    ds.close()


def _problems(count, seed):
    import torch
    rng = np.random.default_rng(seed)
    probs, host = [], []
    for i in range(count):
        n = int(np.exp(rng.uniform(np.log(300), np.log(20000))))
        d = int(rng.integers(2, 9))
        dist = ["uni", "ant", "clu"][i % 3]
        data = make_dataset(dist, n, d, bits=20, seed=seed * 1000 + i)
        k = int(rng.integers(8, 300))
        steps = steps_log(k, 16)
        direction = G.MIN if i % 4 else G.MAX
        cfg = G.plan([G.PART_GRID, G.PART_ANGULAR, G.PART_SLICED, G.PART_NONE][i % 4],
                     slots=4 if i % 5 == 0 else 8, gres_reps=i % 3 == 1)
        probs.append({"data": G.to_device_u32(data),
                      "steps": torch.from_numpy(steps.view(np.int32)).cuda(),
                      "direction": direction, "cfg": cfg})
        host.append((data, steps, direction, cfg))
    return probs, host


def test_batch_matches_single_calls():
    probs, host = _problems(60, seed=5)
    outs, insts, ws = G.batch(probs)
    import torch
    torch.cuda.synchronize()
    for i, ((sky, res, cnt), (data, steps, direction, cfg)) in enumerate(zip(outs, host)):
        S = int(cnt.item())
        ref_sky, ref_res = _compute(data, steps, direction, cfg)
        np.testing.assert_array_equal(sky[:S].cpu().numpy(), ref_sky, err_msg=f"instance {i}")
        np.testing.assert_array_equal(res[:S].cpu().numpy(), ref_res, err_msg=f"instance {i}")
    # a few directly against the oracle
    for i in (0, 7, 13):
        data, steps, direction, cfg = host[i]
        dname = "min" if direction == G.MIN else "max"
        osky = O.skyline_bnl(data, dname)
        exp = O.gres(data, steps, dname, candidates=osky, targets=osky, threads=THREADS)
        S = int(outs[i][2].item())
        np.testing.assert_array_equal(outs[i][1][:S].cpu().numpy(), exp)


def test_batch_graph_capture_and_replay():
    import torch
    probs, host = _problems(24, seed=9)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        outs, insts, ws = G.batch(probs, stream=s)     # warm-up: streams, events, kernel setup
    s.synchronize()
    for sky, res, cnt in outs:
        res.fill_(-7)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        lib = G.load()
        G._check(lib.gres_batch(insts, len(probs), G._ptr(ws), ws.numel(), G._stream_ptr(s)))
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    for (sky, res, cnt), (data, steps, direction, cfg) in zip(outs, host):
        S = int(cnt.item())
        ref_sky, ref_res = _compute(data, steps, direction, cfg)
        np.testing.assert_array_equal(res[:S].cpu().numpy(), ref_res)

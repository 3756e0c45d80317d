"""GPU: the batched and served configurations at their full sizes, against the oracle.

* 512 uneven instances (N log-uniform in [1e3, 2e5], d in 2..8, UNI / ANT / CLU,
  128 log-spaced widths) in one gres_batch call: the exact instance set the
  benchmark times.
* 10,000-query serving set's 64 resident datasets (N log-uniform in [1e3, 2e6],
  d in 2..8): queries on every dataset, each poll result checked directly.

The oracle decides every expected value (Def. 1, Def. 2, Algorithm 1). Where its
skyline costs little (n * S small) it computes the whole skyline and the test
compares it element by element, and gres is checked over that skyline as the
candidate set. On the largest inputs (anticorrelated data at high d, where
nearly every row is a skyline row) the oracle answers sampled rows one by one:
each sampled skyline row must be undominated in r and each sampled other row
dominated (Def. 1), and gres of sampled skyline tuples is computed over all of
r as candidates, which gives the same result as over Sky(r) (stability,
Sec. 3.2).
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2412_02274_gb300 import gres as G

pytestmark = pytest.mark.gpu

THREADS = max(1, os.cpu_count() or 1)
# n * S up to which the oracle's whole skyline is computed
FULL_SKY_BUDGET = 1_000_000_000
# S * S * K up to which gres is checked for every skyline tuple
ALL_TARGETS_BUDGET = 200_000_000
# n * K * targets up to which sampled targets are checked over all of r (at least 8 targets)
SAMPLED_BUDGET = 6_000_000_000


def check_against_oracle(data, direction, sky, res, steps, rng, n_targets=64, n_members=64, cache=None):
    """sky (ascending skyline rows) and res (gres per skyline position) from the GPU,
    against the oracle; returns the number of targets checked. cache: a dict keeping the
    oracle's skyline of `data` between calls."""
    dname = "min" if direction == G.MIN else "max"
    n, S, K = len(data), len(sky), len(steps)
    assert len(res) == S
    assert S >= 1 and np.all(np.diff(sky) > 0) and sky[0] >= 0 and sky[-1] < n
    assert np.all((res >= 0) & (res <= K))
    if n * S <= FULL_SKY_BUDGET:
        if cache is not None and "sky" in cache:
            osky = cache["sky"]
        else:
            osky = O.skyline_threaded(data, dname, THREADS)
            if cache is not None:
                cache["sky"] = osky
        np.testing.assert_array_equal(sky, osky)
        cand = osky
    else:
        n_targets = int(max(8, min(n_targets, SAMPLED_BUDGET // (n * K))))
        pick = rng.choice(S, min(n_members, S), replace=False)
        assert O.skyline_member(data, sky[pick], dname, THREADS).all()
        rest = np.ones(n, bool)
        rest[sky] = False
        others = np.flatnonzero(rest)
        if len(others):
            pick = others[rng.choice(len(others), min(n_members, len(others)), replace=False)]
            assert not O.skyline_member(data, pick, dname, THREADS).any()
        cand = None          # every row of r
    if cand is not None and S * S * K <= ALL_TARGETS_BUDGET:
        pos = np.arange(S)
    else:
        pos = np.unique(np.linspace(0, S - 1, min(n_targets, S)).astype(np.int64))
    exp = O.gres(data, steps, dname, candidates=cand, targets=sky[pos], threads=THREADS)
    np.testing.assert_array_equal(res[pos], exp)
    return len(pos)


def test_batch_512_instances_against_oracle():
    import torch
    import bench
    insts, steps = bench.batch_problems()
    dev = torch.device("cuda")
    tsteps = torch.from_numpy(steps.view(np.int32)).to(dev)
    datas = [G.to_device_u32(data, dev) for _, _, _, data in insts]
    # the benchmark's default plan, and mixed plans (every scheme, 4 / 8 slots)
    probs = [{"data": x, "steps": tsteps, "cfg": G.plan(G.PART_GRID)} for x in datas]
    outs, _, _ = G.batch(probs)
    mixed = [{"data": x, "steps": tsteps,
              "cfg": G.plan([G.PART_GRID, G.PART_ANGULAR, G.PART_SLICED, G.PART_NONE][i % 4],
                            slots=4 if i % 3 == 0 else 8)} for i, x in enumerate(datas)]
    outs_m, _, _ = G.batch(mixed)
    torch.cuda.synchronize()
    rng = np.random.default_rng(4)
    large = 0
    for i, ((dist, n, d, data), (sky, res, cnt), (sky_m, res_m, cnt_m)) in enumerate(zip(insts, outs, outs_m)):
        S = int(cnt.item())
        sky_h, res_h = sky[:S].cpu().numpy(), res[:S].cpu().numpy()
        assert int(cnt_m.item()) == S, f"instance {i}"
        np.testing.assert_array_equal(sky_m[:S].cpu().numpy(), sky_h, err_msg=f"instance {i}")
        np.testing.assert_array_equal(res_m[:S].cpu().numpy(), res_h, err_msg=f"instance {i}")
        try:
            check_against_oracle(data, G.MIN, sky_h, res_h, steps, rng)
        except AssertionError as e:
            raise AssertionError(f"instance {i} ({dist}, n={n}, d={d}, S={S}): {e}") from None
        large += n > 131072
    assert large >= 40      # the >131,072-row path inside the batch is covered


def test_served_queries_against_oracle():
    import bench
    from paper_2412_02274_gb300.inputs import steps_log
    datas = bench.serve_datasets()
    rng = np.random.default_rng(12)
    sv = G.Server(64 << 30, max_batch=128, max_inflight=3)
    ids = [sv.add_dataset(x, G.MIN, G.plan(G.PART_GRID)) for x in datas]
    # one query on every dataset, then a mix of 64 more on random datasets, all in flight at once
    order = list(range(len(ids))) + [int(rng.integers(0, len(ids))) for _ in range(64)]
    queries = [(j, steps_log(int(rng.integers(64, 257)), 16)) for j in order]
    tickets = [sv.submit(ids[j], st) for j, st in queries]
    skies = [sv.sky_idx(i) for i in ids]
    caches = [{} for _ in ids]
    big = 0
    for t, (j, st) in zip(tickets, queries):
        got, _ = sv.poll(t)
        n = len(datas[j])
        try:
            check_against_oracle(datas[j], G.MIN, skies[j], got, st, rng, n_targets=24, n_members=32,
                                 cache=caches[j])
        except AssertionError as e:
            raise AssertionError(f"dataset {j} (n={n}, d={datas[j].shape[1]}, S={len(skies[j])}): {e}") from None
        big += n > 131072
    sv.close()
    assert big >= 20 and max(len(x) for x in datas) > 1_500_000

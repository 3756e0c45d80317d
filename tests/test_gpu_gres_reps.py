"""GPU: Representative Filtering inside the gres stage (GRES_FLAG_GRES_REPS).

The flag only bounds the search by a step at which one of 32 representatives
dominates, so every result must equal the plain search and the oracle.
"""
import os

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2412_02274_gb300 import gres as G
from paper_2412_02274_gb300.inputs import make_dataset, steps_log, steps_linear

pytestmark = pytest.mark.gpu
THREADS = max(1, os.cpu_count() or 1)


def _both(data, steps, direction, scheme, gbits=None):
    x = G.to_device_u32(data)
    out = []
    for reps in (False, True):
        cfg = G.plan(scheme, gres_reps=reps)
        if gbits:
            out.append(G.gres_compute_g(x, gbits, steps, direction, cfg))
        else:
            out.append(G.gres_compute(x, steps, direction, cfg))
    (s0, r0), (s1, r1) = out
    np.testing.assert_array_equal(s0.cpu().numpy(), s1.cpu().numpy())
    np.testing.assert_array_equal(r0.cpu().numpy(), r1.cpu().numpy())
    return s1.cpu().numpy(), r1.cpu().numpy()


def test_same_results_as_the_plain_search_and_the_oracle():
    rng = np.random.default_rng(21)
    for case in range(60):
        d = int(rng.integers(1, 9))
        n = int(rng.integers(1, 400))
        bits = int(rng.choice([4, 8, 12, 20]))
        data = rng.integers(0, 1 << bits, size=(n, d), dtype=np.uint64).astype(np.uint32)
        steps = steps_log(int(rng.integers(1, 80)), bits)
        direction = G.MIN if case % 3 else G.MAX
        scheme = [G.PART_GRID, G.PART_NONE, G.PART_SLICED, G.PART_ANGULAR][case % 4]
        sky, res = _both(data, steps, direction, scheme)
        dname = "min" if direction == G.MIN else "max"
        osky = O.skyline_bnl(data, dname)
        np.testing.assert_array_equal(sky, osky)
        np.testing.assert_array_equal(res, O.gres(data, steps, dname, candidates=osky, targets=osky))
    for dist, n, d, direction in (("ant", 20000, 4, G.MIN), ("uni", 50000, 5, G.MAX), ("clu", 30000, 3, G.MIN)):
        data = make_dataset(dist, n, d, bits=20, seed=7)
        sky, res = _both(data, steps_log(256, 16), direction, G.PART_GRID)
        dname = "min" if direction == G.MIN else "max"
        np.testing.assert_array_equal(res, O.gres(data, steps_log(256, 16), dname, candidates=sky, targets=sky,
                                                  threads=THREADS))
    # the paper's grid parameter form
    data = make_dataset("ant", 20000, 3, bits=20, seed=8)
    _both(data, np.arange(25, 1, -1, dtype=np.uint32), G.MIN, G.PART_GRID, gbits=20)
    # the default workload
    data = make_dataset("ant", 100000, 4, bits=20, seed=0)
    _both(data, steps_log(256, 16), G.MIN, G.PART_GRID)


def test_counters_include_the_representative_tests():
    data = make_dataset("ant", 20000, 4, bits=20, seed=3)
    x = G.to_device_u32(data)
    counts = []
    for reps in (False, True):
        t = torch.zeros(2, dtype=torch.int64, device="cuda")
        G.gres_compute(x, steps_log(256, 16), G.MIN, G.plan(G.PART_GRID, count_tests=True, gres_reps=reps), tests=t)
        counts.append([int(v) for v in t.cpu().tolist()])
    (t0, c0), (t1, c1) = counts
    assert t1 > t0          # the representative tests come on top
    assert c1 <= c0         # the bound never makes the search look at more

"""GPU: the grid-dominance kernel's counters (GRES_FLAG_COUNT_TESTS), which feed the
benchmark's roofline numerator, equal the counts of the CPU restatement of its
search (tests/search_model.py, itself pinned to the oracle) exactly, on small inputs:
every partitioning scheme, both directions, 4 and 8 slots, one and several windows
of widths, skylines of one and of several super-tiles."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2412_02274_gb300 import gres as G
from paper_2412_02274_gb300.inputs import make_dataset, steps_log

from search_model import count_search

pytestmark = pytest.mark.gpu


def _canon(rows, direction):
    r = np.asarray(rows, dtype=np.uint64)
    return (~r & 0xFFFFFFFF) if direction else r


CASES = [
    # dist, n, d, bits, K, scheme, kwargs, slots, direction
    ("ant", 600, 3, 12, 40, G.PART_NONE, {}, 8, G.MIN),
    ("ant", 600, 3, 12, 300, G.PART_NONE, {}, 4, G.MAX),
    ("uni", 3000, 4, 16, 64, G.PART_GRID, {"m": 2}, 8, G.MIN),
    ("ant", 2500, 4, 16, 128, G.PART_GRID, {"m": 3}, 4, G.MIN),
    ("clu", 4000, 5, 16, 96, G.PART_SLICED, {"p": 8}, 8, G.MAX),
    ("ant", 1800, 2, 20, 256, G.PART_ANGULAR, {"m": 4}, 8, G.MIN),
    ("ant", 1800, 5, 14, 64, G.PART_NONE, {}, 8, G.MIN),      # S above 1024: two super-tiles
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}-{c[1]}-d{c[2]}-K{c[4]}-s{c[5]}")
def test_counters_equal_the_search_model(case):
    import torch
    dist, n, d, bits, K, scheme, kw, slots, direction = case
    data = make_dataset(dist, n, d, bits=bits, seed=n + d)
    steps = steps_log(K, bits - 2)
    cfg = G.plan(scheme, slots=slots, count_tests=True, **kw)
    tests = torch.zeros(2, dtype=torch.int64, device="cuda")
    sky, res = G.gres_compute(G.to_device_u32(data), steps, direction, cfg, tests=tests)
    sky = sky.cpu().numpy()
    lane_tests, checks = (int(v) for v in tests.cpu().tolist())
    rows = data[sky]
    if scheme == G.PART_NONE:
        order = np.arange(len(sky))
    else:
        _, order, _ = G.partition(rows, direction, G.plan(scheme, slots=slots, **kw))
        order = order.cpu().numpy().astype(np.int64)
    got, m_tests, m_checks = count_search(_canon(rows[order], direction), steps, direction, slots)
    # the model's results in skyline order are the kernel's (and the oracle's)
    back = np.empty_like(got)
    back[order] = got
    np.testing.assert_array_equal(back, res.cpu().numpy())
    dname = "max" if direction == G.MAX else "min"
    np.testing.assert_array_equal(back, O.gres(data, steps, dname, candidates=sky, targets=sky))
    assert (lane_tests, checks) == (m_tests, m_checks)


@pytest.mark.parametrize("case", CASES[1:6], ids=lambda c: f"{c[0]}-{c[1]}-d{c[2]}-K{c[4]}-s{c[5]}")
def test_per_partition_split_equals_the_search_model(case):
    """GRES_FLAG_COUNT_PARTS: per target partition, the lane-tests and row checks against
    candidates of the same partition and of the others, as the model counts them; the
    lane-tests add up to the total counter."""
    import torch
    dist, n, d, bits, K, scheme, kw, slots, direction = case
    data = make_dataset(dist, n, d, bits=bits, seed=n + d)
    steps = steps_log(K, bits - 2)
    cfg = G.plan(scheme, slots=slots, count_parts=True, **kw)
    P = G.plan_partitions(cfg, d)
    tests = torch.zeros(2 + 4 * P, dtype=torch.int64, device="cuda")
    sky, res = G.gres_compute(G.to_device_u32(data), steps, direction, cfg, tests=tests)
    sky = sky.cpu().numpy()
    t = tests.cpu().numpy()
    split = t[2:].reshape(P, 4)
    rows = data[sky]
    if scheme == G.PART_NONE:
        order, pid = np.arange(len(sky)), np.zeros(len(sky), np.int64)
    else:
        part, order, _ = G.partition(rows, direction, G.plan(scheme, slots=slots, **kw))
        order = order.cpu().numpy().astype(np.int64)
        pid = part.cpu().numpy()[order]
    got, m_tests, m_checks, m_split = count_search(_canon(rows[order], direction), steps, direction, slots,
                                                   pid=pid, nparts=P)
    assert (int(t[0]), int(t[1])) == (m_tests, m_checks)
    np.testing.assert_array_equal(split, m_split)
    assert int(split[:, 0].sum() + split[:, 2].sum()) == int(t[0])

"""GPU: candidate partitioning (Sec. 3.1) and tile minima, bit-exact.

gres_partition runs the partitioning kernels of the gres stage on the
caller's rows. Its partition numbers must equal the oracle's Grid / Angular /
Sliced definitions; the tile order must group partitions in ascending order;
each tile minimum must be the minimum of the tile's canonical rows.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2412_02274_gb300 import gres as G
from paper_2412_02274_gb300.inputs import make_dataset

pytestmark = pytest.mark.gpu


def _canon(data, direction):
    a = data.astype(np.uint64)
    return a if direction == G.MIN else np.uint64(0xFFFFFFFF) - a


def _expected_pid(data, cfg, direction):
    dname = "min" if direction == G.MIN else "max"
    if cfg.scheme == G.PART_GRID:
        return O.grid_pid(data, cfg.m, dname)
    if cfg.scheme == G.PART_ANGULAR:
        return O.angular_pid(data, cfg.m, dname)
    if cfg.scheme == G.PART_SLICED:
        return O.sliced_pid(data, cfg.p, cfg.slice_dim, dname)
    return np.zeros(len(data), np.int64)


def _check(data, cfg, direction, label):
    n, d = data.shape
    part, order, tmin = G.partition(G.to_device_u32(data), direction, cfg)
    part = part.cpu().numpy()
    order = order.cpu().numpy().view(np.uint32).astype(np.int64)
    tmin = tmin.cpu().numpy().view(np.uint32).astype(np.uint64)
    np.testing.assert_array_equal(part, _expected_pid(data, cfg, direction), err_msg=label)
    np.testing.assert_array_equal(np.sort(order), np.arange(n), err_msg=label)
    assert np.all(np.diff(part[order]) >= 0), label
    c = _canon(data, direction)[order]
    T = (n + 31) // 32
    assert tmin.shape == (T, d)
    for t in range(T):
        np.testing.assert_array_equal(tmin[t], c[32 * t: 32 * t + 32].min(axis=0), err_msg=f"{label} tile {t}")


SCHEMES = [
    ("grid-m2", lambda d: G.plan(G.PART_GRID, m=2)),
    ("grid-m4", lambda d: G.plan(G.PART_GRID, m=4)),
    ("grid-m7", lambda d: G.plan(G.PART_GRID, m=7)),
    ("angular-m2", lambda d: G.plan(G.PART_ANGULAR, m=2)),
    ("angular-m5", lambda d: G.plan(G.PART_ANGULAR, m=5)),
    ("angular-m64", lambda d: G.plan(G.PART_ANGULAR, m=64)),
    ("sliced-p1", lambda d: G.plan(G.PART_SLICED, p=1)),
    ("sliced-p16", lambda d: G.plan(G.PART_SLICED, p=16)),
    ("sliced-p64-last", lambda d: G.plan(G.PART_SLICED, p=64, slice_dim=d - 1)),
    ("none", lambda d: G.plan(G.PART_NONE)),
]


@pytest.mark.parametrize("name,mk", SCHEMES, ids=[s[0] for s in SCHEMES])
def test_partition_numbers_match_oracle(name, mk):
    cases = [("uni", 1, 3), ("uni", 2, 2), ("ant", 31, 4), ("clu", 32, 5), ("uni", 33, 1),
             ("ant", 1000, 6), ("clu", 5000, 8), ("uni", 70000, 3), ("ant", 70001, 7),
             ("uni", 150000, 4)]   # above the single-cluster limit: the multi-kernel path
    for i, (dist, n, d) in enumerate(cases):
        data = make_dataset(dist, n, d, bits=20, seed=100 + i)
        cfg = mk(d)
        dims = d if cfg.scheme == G.PART_GRID else d - 1
        if cfg.scheme in (G.PART_GRID, G.PART_ANGULAR) and cfg.m ** max(dims, 0) >= 1 << 32:
            with pytest.raises(G.GresError):      # partition numbers must fit 32 bits
                G.partition(G.to_device_u32(data), G.MIN, cfg)
            continue
        for direction in (G.MIN, G.MAX):
            _check(data, mk(d), direction, f"{name} {dist} n={n} d={d} dir={direction}")


def test_partition_of_a_skyline_and_degenerate_rows():
    # the candidate set gres_compute partitions: the skyline of an ANT dataset
    data = make_dataset("ant", 20000, 4, bits=20, seed=3)
    sky = O.skyline_bnl(data)
    for name, mk in SCHEMES:
        _check(data[sky], mk(4), G.MIN, f"skyline {name}")
    # identical rows (zero span, all angles zero), a single distinct value per attribute
    same = np.full((100, 3), 12345, np.uint32)
    zero = np.zeros((40, 5), np.uint32)
    for name, mk in SCHEMES:
        _check(same, mk(3), G.MIN, f"identical {name}")
        _check(zero, mk(5), G.MAX, f"zeros {name}")
    # full 32-bit values (spans of 2^32)
    rng = np.random.default_rng(1)
    wide = rng.integers(0, 1 << 32, size=(3000, 4), dtype=np.uint64).astype(np.uint32)
    wide[0] = 0
    wide[1] = 0xFFFFFFFF
    for name, mk in SCHEMES:
        _check(wide, mk(4), G.MIN, f"wide {name}")

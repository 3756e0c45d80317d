"""GPU: the paper's grid-parameter form (projection floor(v g / 2^B)), bit-exact.

gres_compute_g against the oracle's g-list form (Algorithm 1 with the paper's
g scan). The oracle reports the g value at which a tuple leaves (1 = never);
the library reports its index in the list (len = never).
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2412_02274_gb300 import gres as G
from paper_2412_02274_gb300.inputs import make_dataset, steps_log

pytestmark = pytest.mark.gpu


def _expected_idx(data, bits, glist, direction):
    dname = "min" if direction == G.MIN else "max"
    sky = O.skyline_bnl(data, dname)
    gv = O.gres_glist(data, bits, glist, dname, candidates=sky, targets=sky).view(np.uint32)
    pos = {int(g): i for i, g in enumerate(glist)}
    assert 1 not in pos
    return sky, np.array([pos.get(int(v), len(glist)) for v in gv], dtype=np.int32)


def _check(data, bits, glist, direction=G.MIN, cfg=None, label=""):
    sky, idx = G.gres_compute_g(G.to_device_u32(data), bits, glist, direction, cfg)
    esky, eidx = _expected_idx(data, bits, glist, direction)
    np.testing.assert_array_equal(sky.cpu().numpy(), esky, err_msg=label)
    np.testing.assert_array_equal(idx.cpu().numpy(), eidx, err_msg=label)


def test_tiny_random_against_the_oracle():
    rng = np.random.default_rng(17)
    for case in range(120):
        bits = int(rng.choice([3, 4, 6, 8, 12]))
        d = int(rng.integers(1, 9))
        n = int(rng.integers(1, 60))
        hi = 1 << bits if case % 4 else 1 << min(bits + 3, 32)   # some values above 2^B - 1
        data = rng.integers(0, hi, size=(n, d), dtype=np.uint64).astype(np.uint32)
        gmax = int(rng.integers(2, 3 * (1 << bits)))
        glist = np.sort(rng.choice(np.arange(2, gmax + 2), size=min(gmax, int(rng.integers(1, 40))),
                                   replace=False))[::-1].astype(np.uint32)
        direction = G.MIN if case % 3 else G.MAX
        cfg = G.plan([G.PART_GRID, G.PART_NONE, G.PART_SLICED, G.PART_ANGULAR][case % 4], slots=4 if case % 5 == 0 else 8)
        _check(data, bits, glist, direction, cfg, label=f"case {case}")


def test_paper_practical_g_bar_25_and_exact_g_bar():
    # Algorithm 1 with the practical g_bar = 25 (g = 25 .. 2) on 20-bit ANT and CLU data
    for dist, n, d in (("ant", 20000, 4), ("clu", 30000, 3)):
        data = make_dataset(dist, n, d, bits=20, seed=4)
        _check(data, 20, np.arange(25, 1, -1, dtype=np.uint32), G.MIN, label=f"{dist} g_bar=25")
    # the exact g_bar = floor(2^B / l) on a small set (every finer grid changes nothing)
    data = make_dataset("uni", 3000, 3, bits=12, seed=5)
    l = O.min_gap(data)
    g_bar = (1 << 12) // l
    glist = np.arange(g_bar, 1, -1, dtype=np.uint32)
    _check(data, 12, glist, G.MIN, label="exact g_bar")
    _check(data, 12, glist, G.MAX, label="exact g_bar max")


def test_divisors_of_two_to_the_b_equal_the_width_form():
    data = make_dataset("ant", 40000, 5, bits=20, seed=6)
    gl = np.array([1 << 14, 1 << 12, 1 << 10, 512, 64, 16, 4, 2], dtype=np.uint32)
    widths = ((1 << 20) // gl).astype(np.uint32)
    for direction in (G.MIN, G.MAX):
        sky_g, idx_g = G.gres_compute_g(G.to_device_u32(data), 20, gl, direction)
        sky_w, idx_w = G.gres_compute(G.to_device_u32(data), widths, direction)
        np.testing.assert_array_equal(sky_g.cpu().numpy(), sky_w.cpu().numpy())
        np.testing.assert_array_equal(idx_g.cpu().numpy(), idx_w.cpu().numpy())


def test_full_range_values_and_32_bits():
    rng = np.random.default_rng(3)
    data = rng.integers(0, 1 << 32, size=(400, 3), dtype=np.uint64).astype(np.uint32)
    data[:4] = [[0, 0xFFFFFFFF, 7], [0xFFFFFFFF, 0, 0xFFFFFFFE], [0x80000000, 0x7FFFFFFF, 1], [1, 1, 0xFFFFFFFF]]
    glist = np.array([4000000000, 3000000001, 65537, 1000, 3, 2], dtype=np.uint32)
    for direction in (G.MIN, G.MAX):
        _check(data, 32, glist, direction, label=f"32-bit dir={direction}")
    with pytest.raises(G.GresError):
        G.gres_compute_g(G.to_device_u32(data), 33, glist)
    with pytest.raises(G.GresError):
        G.gres_compute_g(G.to_device_u32(data), 20, glist[::-1].copy())

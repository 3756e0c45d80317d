"""Pins for the CPU oracle: each check ties it to something other than itself.

* hand-derived cases (tests/golden/hand_cases.txt) and the paper's Grid example
  (Sec. 3.1, tests/golden/grid_example_m3d2.txt);
* brute force on tiny inputs: the pairwise form of Def. 2 (over r and over
  Sky(r)) against the literal set form of Algorithm 1, which builds the
  projected relation as a set and computes its skyline;
* invariants the paper states or implies: stability (Sec. 3.2), no exit at
  widths up to the smallest non-zero gap l (Sec. 3.2), the sentinel for tuples
  that never leave (Def. 2), direction symmetry (Sec. 2), permutation
  invariance, the paper's g form equal to the width form when g divides 2^B;
* skylines against the textbook 2-D staircase sweep and the expected number of
  maxima of uniform points (a closed-form recurrence).
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2412_02274_gb300.inputs import make_dataset, steps_log, steps_linear

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _hand_cases():
    cases = []
    with open(os.path.join(GOLDEN, "hand_cases.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            direction, steps, rows, expect = [x.strip() for x in line.split("|")]
            rows = np.array([[int(v) for v in r.split()] for r in rows.split(";")], np.uint32)
            cases.append((direction, np.array(steps.split(), np.uint32), rows,
                          np.array(expect.split(), np.int32)))
    return cases


@pytest.mark.parametrize("case", _hand_cases(), ids=lambda c: f"{c[0]}-{len(c[2])}rows")
def test_hand_cases(case):
    direction, steps, rows, expect = case
    sky, res = O.gres_all(rows, steps, direction)
    assert list(res) == list(expect)
    lit = O.gres_literal(rows, steps, direction, targets=sky)
    assert list(lit) == list(expect)


def test_paper_grid_example():
    """Sec. 3.1: with m=3, d=2, partition 1 grid-dominates exactly partitions 5 and 8."""
    spec = {}
    with open(os.path.join(GOLDEN, "grid_example_m3d2.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, *v = line.split()
            spec[k] = [int(x) for x in v]
    m, d, cell = spec["m"][0], spec["d"][0], spec["cell"][0]
    got = [h for h in range(m ** d) if O.cell_grid_dominates(cell, h, d, m)]
    assert got == spec["dominated"]
    # The partition-number formula places a point of cell (c1, c2) in partition c1 + 3 c2:
    # values 0..8 span three slices of width 3 per dimension.
    pts = np.array([[0, 0], [8, 8], [4, 1], [7, 4], [6, 8], [2, 5]], np.uint32)
    assert list(O.grid_pid(pts, 3)) == [0, 8, 1, 5, 8, 3]


def test_dominance_definition():
    assert O.dominates([1, 2], [1, 3])
    assert not O.dominates([1, 3], [1, 3])          # equal tuples do not dominate
    assert not O.dominates([0, 4], [1, 3])          # incomparable
    assert O.dominates([2, 3], [1, 3], "max")
    assert not O.dominates([1, 3], [2, 3], "max")


def _tiny(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 20))
    d = int(rng.integers(1, 5))
    bits = int(rng.integers(1, 6))
    data = rng.integers(0, 1 << bits, size=(n, d), dtype=np.uint32)
    return data, bits


@pytest.mark.parametrize("direction", ["min", "max"])
def test_brute_force_tiny_all_variants(direction):
    """P1: pairwise over r, pairwise over Sky(r) and the literal set form agree, every width."""
    for seed in range(300):
        data, bits = _tiny(seed)
        steps = np.arange(1, (1 << bits) + 2, dtype=np.uint32)
        sky = O.skyline_bnl(data, direction)
        assert list(sky) == list(O.skyline_allpairs(data, direction))
        over_r = O.gres(data, steps, direction, candidates=None, targets=sky)
        over_sky = O.gres(data, steps, direction, candidates=sky, targets=sky)
        lit = O.gres_literal(data, steps, direction, targets=sky)
        assert list(over_r) == list(over_sky) == list(lit), seed


def test_finest_widths_never_exit():
    """P2 (Sec. 3.2): widths up to l, the smallest non-zero gap, create no new dominance."""
    for seed in range(40):
        data = make_dataset("ant", 300, 3, bits=12, seed=seed)
        gap = O.min_gap(data)
        assert gap >= 1
        steps = np.arange(1, gap + 1, dtype=np.uint32)
        sky, res = O.gres_all(data, steps)
        assert (res == len(steps)).all()
    # width 1 is the identity: every skyline tuple stays
    data = make_dataset("uni", 2000, 4, bits=20, seed=3)
    sky, res = O.gres_all(data, np.array([1], np.uint32))
    assert (res == 1).all()


def test_stability_over_r_and_sky():
    """P3 (Sec. 3.2): gres is the same with all of r or with Sky(r) as candidates."""
    for dist, seed in [("uni", 0), ("ant", 1), ("clu", 2), ("ant", 3)]:
        data = make_dataset(dist, 600, 3, bits=16, seed=seed)
        steps = steps_log(48, 12)
        sky = O.skyline_bnl(data)
        a = O.gres(data, steps, candidates=None, targets=sky)
        b = O.gres(data, steps, candidates=sky, targets=sky)
        assert (a == b).all()


def test_sentinels_and_collapse():
    """P4: N=1 never leaves; identical rows all stay; widths >= 2^B collapse everything."""
    one = np.array([[5, 6, 7]], np.uint32)
    assert list(O.gres_all(one, np.array([1, 2, 3], np.uint32))[1]) == [3]
    same = np.tile(np.array([[3, 9]], np.uint32), (7, 1))
    sky, res = O.gres_all(same, np.array([1, 2, 5], np.uint32))
    assert list(sky) == list(range(7)) and (res == 3).all()
    data = make_dataset("uni", 500, 3, bits=10, seed=5)
    sky, res = O.gres_all(data, np.array([1 << 10, 1 << 11], np.uint32))
    assert (res == 2).all()
    # a row holding the minimum of every attribute never leaves
    data = make_dataset("uni", 300, 3, bits=10, seed=6)
    data[17] = data.min(axis=0)
    sky, res = O.gres_all(data, steps_log(32, 10))
    assert list(sky) == [17] and list(res) == [32]


def test_direction_symmetry():
    """P6 (Sec. 2): larger-is-better on v equals smaller-is-better on 2^B-1-v for widths dividing 2^B."""
    bits = 12
    steps = np.array([1, 2, 4, 16, 64, 256, 1024], np.uint32)
    for seed in range(5):
        data = make_dataset("ant", 400, 3, bits=bits, seed=seed)
        flipped = ((1 << bits) - 1 - data).astype(np.uint32)
        s1, r1 = O.gres_all(data, steps, "max")
        s2, r2 = O.gres_all(flipped, steps, "min")
        assert list(s1) == list(s2) and list(r1) == list(r2)


def test_permutation_invariance():
    """P7: shuffling rows permutes the skyline and keeps every tuple's gres."""
    data = make_dataset("clu", 800, 3, bits=14, seed=9)
    steps = steps_log(40, 12)
    s1, r1 = O.gres_all(data, steps)
    perm = np.random.default_rng(0).permutation(len(data))
    s2, r2 = O.gres_all(data[perm], steps)
    m1 = dict(zip(s1.tolist(), r1.tolist()))
    m2 = {int(perm[i]): v for i, v in zip(s2.tolist(), r2.tolist())}
    assert m1 == m2


def test_gmode_equals_width_mode():
    """P8: floor(x g / 2^B) = floor(x / (2^B / g)) when g divides 2^B, so both forms agree."""
    bits = 10
    gl = [512, 256, 128, 64, 32, 16, 8, 4, 2]
    widths = np.array([(1 << bits) // g for g in gl], np.uint32)
    for seed in range(6):
        data = make_dataset("ant", 300, 3, bits=bits, seed=seed)
        sky = O.skyline_bnl(data)
        gm = O.gres_glist(data, bits, gl, candidates=sky, targets=sky)
        wm = O.gres(data, widths, candidates=sky, targets=sky)
        exp = np.array([gl[k] if k < len(gl) else 1 for k in wm], np.int32)
        assert (gm == exp).all()
    # Algorithm 1 literally, with g_bar from l (Sec. 3.2): no tuple leaves at g > g_bar
    data = make_dataset("uni", 200, 2, bits=8, seed=1)
    gbar = (1 << 8) // O.min_gap(data)
    sky = O.skyline_bnl(data)
    full = O.gres_glist(data, 8, np.arange(4 * gbar, 1, -1), candidates=sky, targets=sky)
    assert (full <= gbar).all()
    assert (O.gres_gmode(data, 8, gbar, candidates=sky, targets=sky) == full).all()


def test_gproj_floor():
    v = np.array([0, 1, 63, 64, 65, 127, 128, 0xFFFFFFFF], np.uint32)
    assert list(O.gproj(v, 64)) == [0, 0, 0, 1, 1, 1, 2, 67108863]


def _staircase_2d(data):
    """Textbook 2-D maxima sweep (smaller is better): sort by (x, y), keep strict y records."""
    order = sorted(range(len(data)), key=lambda i: (int(data[i, 0]), int(data[i, 1])))
    out, best_y, prev = [], None, None
    for i in order:
        x, y = int(data[i, 0]), int(data[i, 1])
        if prev is not None and (x, y) == prev:
            if out and (int(data[out[-1], 0]), int(data[out[-1], 1])) == (x, y):
                out.append(i)        # duplicate of a kept point
            continue
        if best_y is None or y < best_y:
            out.append(i)
            best_y = y
        prev = (x, y)
    return sorted(out)


def test_skyline_2d_staircase_and_1d():
    for seed in range(20):
        data = make_dataset("uni", 500, 2, bits=6, seed=seed)    # many ties
        assert list(O.skyline_bnl(data)) == _staircase_2d(data)
    data = np.array([[3], [1], [2], [1]], np.uint32)
    assert list(O.skyline_bnl(data)) == [1, 3]


def test_skyline_member_row_by_row():
    """Def. 1 asked row by row (the oracle's check for inputs too large for its BNL): on every
    row it is the 2-D staircase and the BNL skyline, in both directions, with one thread or
    many; on a sample of rows it answers each row as on the whole input."""
    for seed in range(12):
        data = make_dataset("uni", 400, 2, bits=6, seed=seed)
        assert list(O.skyline_threaded(data, threads=1)) == _staircase_2d(data)
        assert list(O.skyline_threaded(data, threads=4)) == _staircase_2d(data)
    for dist, d in (("ant", 3), ("clu", 5), ("uni", 8), ("ant", 1)):
        data = make_dataset(dist, 1500, d, bits=8, seed=d)
        for direction in ("min", "max"):
            full = O.skyline_member(data, direction=direction, threads=3)
            assert list(np.flatnonzero(full)) == list(O.skyline_bnl(data, direction))
            rows = np.array([0, 7, 7, 1499, 311, 42], np.int64)
            assert list(O.skyline_member(data, rows, direction)) == list(full[rows])
    # duplicates of a skyline row stay in it; a row strictly inside is out
    data = np.array([[1, 2], [1, 2], [2, 3], [0, 5]], np.uint32)
    assert list(O.skyline_member(data)) == [True, True, False, True]


def test_planted_skyline_construction():
    """The planted construction (plane rows plus dominated offsets) has the plane rows as its
    skyline: checked against both oracle skylines, so the large GPU tests that rely on it
    rest on a pinned expectation."""
    from planted import planted_skyline
    for d, seed in ((2, 0), (5, 1), (8, 2)):
        data, sky = planted_skyline(1500, 1200, d, seed=seed)
        assert list(O.skyline_bnl(data)) == list(sky)
        assert list(O.skyline_allpairs(data)) == list(sky)


def _expected_maxima(n, d):
    a = np.ones(n + 1)
    a[0] = 0.0
    for _ in range(2, d + 1):
        k = np.arange(1, n + 1)
        b = np.zeros(n + 1)
        b[1:] = np.cumsum(a[1:] / k)
        a = b
    return a[n]


def test_uniform_skyline_size_matches_expected_maxima():
    """P10: mean skyline size of uniform data against the expected number of maxima."""
    n, d = 3000, 3
    sizes = [len(O.skyline_bnl(make_dataset("uni", n, d, bits=30, seed=s))) for s in range(24)]
    exp = _expected_maxima(n, d)
    assert abs(np.mean(sizes) - exp) / exp < 0.2, (np.mean(sizes), exp)


def test_sliced_sizes_and_angular_bins():
    """Sec. 3.1: Sliced slices differ in size by at most one; Angular bins follow atan2."""
    data = make_dataset("uni", 1003, 3, bits=16, seed=2)
    for p in (1, 7, 64, 2000):
        pid = O.sliced_pid(data, p)
        counts = np.bincount(pid, minlength=p)
        assert counts.max() - counts.min() <= 1
        order = np.lexsort((np.arange(len(data)), data[:, 0]))
        assert (np.diff(pid[order]) >= 0).all()
    rng = np.random.default_rng(4)
    pts = rng.integers(0, 1 << 20, size=(4000, 3), dtype=np.uint32)
    pts[0] = 0
    for m in (2, 3, 4):
        pid = O.angular_pid(pts, m)
        x = pts.astype(np.float64) - pts.min(axis=0)
        exp = np.zeros(len(pts), np.int64)
        near = np.zeros(len(pts), bool)
        for i in range(2):
            phi = np.arctan2(np.sqrt((x[:, i + 1:] ** 2).sum(1)), x[:, i])
            u = 2 * phi * m / np.pi
            near |= np.abs(u - np.round(u)) < 1e-9
            exp += np.minimum(np.floor(u), m - 1).astype(np.int64) * m ** i
        ok = ~near
        assert ok.sum() > 3900
        assert (pid[ok] == exp[ok]).all()


def test_step_generators():
    s = steps_log(256, 16)
    assert len(s) == 256 and s[0] == 1 and s[-1] == 65536 and (np.diff(s.astype(np.int64)) > 0).all()
    prev = 0
    for v in s.tolist():
        top6 = v < 64 or (v >> (v.bit_length() - 6)) << (v.bit_length() - 6) == v
        assert top6 or v == prev + 1
        prev = v
    lin = steps_linear(64, 64)
    assert lin[0] == 64 and lin[-1] == 4096

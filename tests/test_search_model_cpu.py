"""The CPU restatement of the grid-dominance search (tests/search_model.py) is exact:
on tiny random inputs its first exit step of every skyline tuple equals the
oracle's (Def. 2 over Sky(r), both directions, one and several windows of
widths). That makes its counts a faithful reference for the kernel's counters
(tests/test_gpu_counters.py)."""
import numpy as np

from oracle import oracle as O
from paper_2412_02274_gb300.inputs import make_dataset, steps_log

from search_model import count_search


def _canon(rows, direction):
    r = np.asarray(rows, dtype=np.uint64)
    return (~r & 0xFFFFFFFF) if direction else r


def test_model_matches_oracle_on_tiny_inputs():
    rng = np.random.default_rng(6)
    for case in range(24):
        d = int(rng.integers(1, 6))
        n = int(rng.integers(5, 140))
        direction = case % 2
        bits = int(rng.integers(6, 13))
        data = rng.integers(0, 1 << bits, size=(n, d)).astype(np.uint32)
        if case % 3 == 0:
            data = make_dataset("ant", n, max(d, 2), bits=bits, seed=case)
            d = data.shape[1]
        k = int(rng.integers(1, 90))
        steps = np.unique(rng.integers(1, 1 << bits, size=k)).astype(np.uint32)
        dname = "max" if direction else "min"
        sky = O.skyline_bnl(data, dname)
        exp = O.gres(data, steps, dname, candidates=sky, targets=sky)
        for slots in (4, 8):
            got, tests, checks = count_search(_canon(data[sky], direction), steps, direction, slots)
            np.testing.assert_array_equal(got, exp, err_msg=f"case {case} slots {slots}")
            assert tests % 32 == 0 and checks % 32 == 0 and checks >= 32 * len(sky)


def test_model_counts_a_hand_case():
    """Two skyline tuples s = (2, 5), t = (3, 4), widths 1..6 (smaller is better): t leaves
    at width 3, s at width 5. One tile and one super-tile, eight slots, one window:
    per target 3 checks (super-tile, tile, rows) and the tests of the one candidate
    that can matter."""
    rows = np.array([[2, 5], [3, 4]], np.uint64)
    got, tests, checks = count_search(rows, [1, 2, 3, 4, 5, 6], 0, 8)
    assert list(got) == [4, 2]
    assert checks == 2 * 3 * 32
    # each target tests the other once, in slot 0 (excess 1 < width of best-1 = 6)
    assert tests == 2 * 32

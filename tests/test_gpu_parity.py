"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, bit-exact.

Every result here is an integer (skyline row numbers, step indices, grid
projections), so the bar is exact equality, element by element.
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2412_02274_gb300 import gres as G
from paper_2412_02274_gb300.inputs import make_dataset, steps_log, steps_linear

pytestmark = pytest.mark.gpu

THREADS = max(1, os.cpu_count() or 1)
SCHEMES = [G.PART_NONE, G.PART_GRID, G.PART_ANGULAR, G.PART_SLICED]


def _gpu(data, steps, direction=G.MIN, cfg=None):
    t = G.to_device_u32(data)
    sky, res = G.gres_compute(t, steps, direction, cfg)
    return sky.cpu().numpy(), res.cpu().numpy()


def _oracle(data, steps, direction="min"):
    sky = O.skyline_bnl(data, direction)
    res = O.gres(data, steps, direction, candidates=sky, targets=sky, threads=THREADS)
    return sky, res


def _check(data, steps, direction=G.MIN, cfg=None, oracle=None):
    gs, gr = _gpu(data, steps, direction, cfg)
    osky, ores = oracle if oracle is not None else _oracle(data, steps, "min" if direction == G.MIN else "max")
    np.testing.assert_array_equal(gs, osky)
    np.testing.assert_array_equal(gr, ores)
    return gs, gr


def test_hand_cases():
    from tests.test_oracle_pins import _hand_cases
    for direction, steps, rows, expect in _hand_cases():
        gs, gr = _gpu(rows, steps, G.MIN if direction == "min" else G.MAX)
        assert list(gr) == list(expect)


def test_tiny_random():
    """Brute force on tiny inputs: every dimensionality, both directions, all schemes."""
    rng = np.random.default_rng(123)
    for case in range(240):
        n = int(rng.integers(1, 70))
        d = int(rng.integers(1, 9))
        bits = int(rng.integers(1, 7))
        data = rng.integers(0, 1 << bits, size=(n, d), dtype=np.uint32)
        cand = np.arange(1, (1 << bits) + 3)
        steps = np.sort(rng.choice(cand, size=int(rng.integers(1, len(cand) + 1)), replace=False))
        direction = G.MIN if case % 2 == 0 else G.MAX
        cfg = G.plan(SCHEMES[case % 4], slots=4 if case % 3 == 0 else 8)
        _check(data, steps, direction, cfg)


@pytest.mark.parametrize("seed", range(5))
def test_uniform_1k_2d(seed):
    """N=1,000, d=2, values in [0, 2^16), widths 64, 128, ..., 4096: full parity."""
    data = make_dataset("uni", 1000, 2, bits=16, seed=seed)
    _check(data, steps_linear(64, 64))


@pytest.mark.parametrize("scheme", SCHEMES)
def test_anticorrelated_small(scheme):
    """ANT N=5,000, d=4, 256 log-spaced widths: several tiles and a ragged tail."""
    data = make_dataset("ant", 5000, 4, bits=20, seed=1)
    _check(data, steps_log(256, 16), G.MIN, G.plan(scheme, m=4))


@pytest.mark.parametrize("scheme", SCHEMES)
def test_uniform_small_6d(scheme):
    data = make_dataset("uni", 50000, 6, bits=20, seed=2)
    _check(data, steps_log(256, 16), G.MIN, G.plan(scheme, m=2, p=64))


def test_clustered_and_max_direction():
    data = make_dataset("clu", 20000, 5, bits=20, seed=3)
    _check(data, steps_log(128, 16), G.MAX, G.plan(G.PART_GRID))
    _check(data, steps_log(128, 16), G.MIN, G.plan(G.PART_SLICED, p=16, slice_dim=3))


def test_full_size_anticorrelated_100k():
    """ANT N=100,000, d=4, 256 widths, Grid m=4: every skyline tuple against the oracle."""
    data = make_dataset("ant", 100000, 4, bits=20, seed=0)
    oracle = _oracle(data, steps_log(256, 16))
    _check(data, steps_log(256, 16), G.MIN, G.plan(G.PART_GRID, m=4), oracle=oracle)


def test_full_size_uniform_1m():
    """UNI N=1,000,000, d=6, 256 widths: every skyline tuple, Angular / Sliced / no pruning."""
    data = make_dataset("uni", 1000000, 6, bits=20, seed=0)
    steps = steps_log(256, 16)
    oracle = _oracle(data, steps)
    for cfg in (G.plan(G.PART_ANGULAR, m=2), G.plan(G.PART_SLICED, p=64), G.plan(G.PART_NONE)):
        _check(data, steps, G.MIN, cfg, oracle=oracle)


def test_edge_cases():
    # empty input
    gs, gr = _gpu(np.zeros((0, 3), np.uint32), [1, 2])
    assert len(gs) == 0 and len(gr) == 0
    # single row, one step
    gs, gr = _gpu(np.array([[7, 7]], np.uint32), [3])
    assert list(gs) == [0] and list(gr) == [1]
    # identical rows: all in the skyline, none ever leaves
    gs, gr = _gpu(np.full((100, 4), 12345, np.uint32), steps_log(64, 16))
    assert list(gs) == list(range(100)) and (gr == 64).all()
    # values and widths near the top of uint32 (cell bounds that overflow 32 bits)
    rng = np.random.default_rng(5)
    data = (0xFFFFFFFF - rng.integers(0, 1 << 12, size=(3000, 3))).astype(np.uint32)
    steps = np.array([1, 5, 1000, 1 << 20, (1 << 31) + 7, 0xFFFFFFFE, 0xFFFFFFFF], np.uint32)
    for direction in (G.MIN, G.MAX):
        _check(data, steps, direction)
    data = rng.integers(0, 1 << 12, size=(3000, 3)).astype(np.uint32)
    for direction in (G.MIN, G.MAX):
        _check(data, steps, direction)
    # more steps than one register window (K > 256), K not a multiple of 32
    data = make_dataset("ant", 3000, 3, bits=20, seed=7)
    _check(data, np.arange(1, 601, dtype=np.uint32) * 37)
    # d = 1 and d = 8
    _check(make_dataset("uni", 5000, 1, bits=10, seed=1), steps_log(40, 10))
    _check(make_dataset("ant", 4000, 8, bits=20, seed=1), steps_log(128, 16))


@pytest.mark.parametrize("n", [16000, 40000])
def test_large_skyline_streams_from_global_memory(n):
    """Skylines too large for shared memory (d=2, every row on one anti-diagonal); the
    40,000-row case also takes the multi-block sorts (more than 16,384 survivors)."""
    x = np.arange(n, dtype=np.uint32) * 23
    data = np.stack([x, x.max() - x], axis=1).astype(np.uint32)
    data = data[np.random.default_rng(n).permutation(n)]
    steps = steps_log(48, 20)
    gs, gr = _gpu(data, steps, G.MIN, G.plan(G.PART_GRID))
    assert list(gs) == list(range(n))
    assert list(O.skyline_allpairs(data[:2000])) == list(range(2000))
    targets = np.linspace(0, n - 1, 97).astype(np.int64)
    exp = O.gres(data, steps, candidates=np.arange(n), targets=targets, threads=THREADS)
    np.testing.assert_array_equal(gr[targets], exp)


@pytest.mark.parametrize("d,n_plane,n_dom,direction", [(5, 150000, 100000, G.MIN), (6, 200000, 150000, G.MIN),
                                                      (8, 120000, 100000, G.MIN), (7, 140000, 60000, G.MAX)])
def test_large_path_many_survivors(d, n_plane, n_dom, direction):
    """More than 131,072 filter survivors on the multi-kernel path (finer survivor keys, up to
    four digit passes): the planted skyline exactly, and gres of sampled skyline tuples
    against the oracle over the whole skyline. Larger-is-better takes the planted data
    mirrored inside 20 bits (v -> 2^20 - 1 - v), which keeps the same skyline rows."""
    from planted import planted_skyline
    data, sky = planted_skyline(n_plane, n_dom, d, seed=d)
    if direction == G.MAX:
        assert int(data.max()) < (1 << 20)
        data = ((1 << 20) - 1 - data).astype(np.uint32)
    steps = steps_log(32, 16)
    gs, gr = _gpu(data, steps, direction, G.plan(G.PART_GRID))
    np.testing.assert_array_equal(gs, sky)
    pick = np.linspace(0, len(sky) - 1, 61).astype(np.int64)
    exp = O.gres(data, steps, "min" if direction == G.MIN else "max", candidates=sky, targets=sky[pick],
                 threads=THREADS)
    np.testing.assert_array_equal(gr[pick], exp)


def test_gproj_exhaustive_20bit():
    """gproj with multiply-high division equals floor division for every v < 2^20."""
    v = np.arange(1 << 20, dtype=np.uint32)
    tv = G.to_device_u32(v)
    for steps in (steps_log(256, 16), steps_linear(64, 64)):
        out = G.gproj(tv, steps).cpu().numpy().view(np.uint32)
        for j, delta in enumerate(steps.tolist()):
            np.testing.assert_array_equal(out[j], O.gproj(v, delta))


def test_gproj_full_range_edges():
    rng = np.random.default_rng(11)
    deltas = np.unique(np.concatenate([rng.integers(1, 1 << 32, size=200, dtype=np.uint64),
                                       [1, 2, 3, 7, 641, 65535, 65536, 1 << 31, (1 << 31) + 1,
                                        0xFFFFFFFE, 0xFFFFFFFF]])).astype(np.uint32)
    v = np.concatenate([rng.integers(0, 1 << 32, size=100000, dtype=np.uint64),
                        [0, 1, 0xFFFFFFFF, 0xFFFFFFFE, 1 << 31, (1 << 31) - 1]]).astype(np.uint32)
    # multiples of each delta and their neighbours
    extra = []
    for dlt in deltas[:64].astype(np.uint64):
        for q in (1, 2, 3, 1000):
            x = dlt * np.uint64(q)
            if x < (1 << 32):
                extra += [int(x) - 1, int(x), min(int(x) + 1, 0xFFFFFFFF)]
    v = np.concatenate([v, np.array(extra, np.uint64).astype(np.uint32)])
    out = G.gproj(G.to_device_u32(v), deltas).cpu().numpy().view(np.uint32)
    for j, delta in enumerate(deltas.tolist()):
        np.testing.assert_array_equal(out[j], O.gproj(v, delta))


def test_host_buffer_entry_and_counts():
    data = make_dataset("ant", 20000, 4, bits=20, seed=4)
    steps = steps_log(256, 16)
    osky, ores = _oracle(data, steps)
    hs, hr = G.gres_compute_host(data, steps, G.MIN, G.plan(G.PART_GRID, m=4))
    np.testing.assert_array_equal(hs, osky)
    np.testing.assert_array_equal(hr, ores)
    import torch
    tests = torch.zeros(2, dtype=torch.int64, device="cuda")
    G.gres_compute(G.to_device_u32(data), steps, G.MIN, G.plan(G.PART_GRID, m=4, count_tests=True),
                   tests=tests)
    executed, checks = (int(v) for v in tests.cpu().tolist())
    S = len(osky)
    assert 0 < executed <= S * 32 * S * 256 and checks > 0


def test_sky_compute_only():
    data = make_dataset("clu", 30000, 3, bits=20, seed=9)
    sky = G.sky_compute(G.to_device_u32(data)).cpu().numpy()
    np.testing.assert_array_equal(sky, O.skyline_bnl(data))
    sky = G.sky_compute(G.to_device_u32(data), G.MAX).cpu().numpy()
    np.testing.assert_array_equal(sky, O.skyline_bnl(data, "max"))


def test_graph_capture_replay():
    """With no host count the whole call queues without a host wait and can be graph-captured."""
    import torch
    data = make_dataset("ant", 20000, 4, bits=20, seed=6)
    steps = steps_log(256, 16)
    t = G.to_device_u32(data)
    ws = G.alloc_workspace(len(data), 4, len(steps))
    cfg = G.plan(G.PART_GRID, m=4)
    out = (torch.empty(len(data), dtype=torch.int64, device="cuda"),
           torch.empty(len(data), dtype=torch.int32, device="cuda"),
           torch.zeros(1, dtype=torch.int64, device="cuda"))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        G.gres_compute(t, steps, G.MIN, cfg, ws=ws, stream=s, sync=False, out=out)  # warm-up
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    out[1].fill_(-1)
    with torch.cuda.graph(g, stream=s):
        G.gres_compute(t, steps, G.MIN, cfg, ws=ws, stream=s, sync=False, out=out)
    g.replay()
    torch.cuda.synchronize()
    S = int(out[2].item())
    osky, ores = _oracle(data, steps)
    np.testing.assert_array_equal(out[0][:S].cpu().numpy(), osky)
    np.testing.assert_array_equal(out[1][:S].cpu().numpy(), ores)

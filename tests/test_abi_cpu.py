"""Host-side checks of the C ABI: no GPU needed (no kernel is launched here)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2412_02274_gb300 import gres as G
from paper_2412_02274_gb300.inputs import steps_log, steps_linear

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(",
                            src, flags=re.M)
    return sorted(set(names))


def test_library_builds_loads_and_exports_every_declared_symbol():
    lib = G.load()
    names = _declared_functions()
    assert "gres_compute" in names and "sky_compute" in names and "gres_gproj" in names
    for name in names:
        assert hasattr(lib, name), f"libgres does not export {name}"
    assert "sm_103a" in G.version()


def test_workspace_size_and_validation():
    assert G.workspace_size(1000, 2, 64) > 0
    assert G.workspace_size(0, 3, 1) > 0
    assert G.workspace_size(10**6, 6, 256) > G.workspace_size(10**5, 6, 256)
    assert G.workspace_size(1000, 4, 64, host=True) > G.workspace_size(1000, 4, 64)
    for bad in [(10, 0, 5), (10, 9, 5), (-1, 2, 5), (10, 2, 0)]:
        with pytest.raises(G.GresError) as e:
            G.workspace_size(*bad)
        assert e.value.status == 1


def test_invalid_arguments_are_rejected_before_any_launch():
    lib = G.load()
    fake = ctypes.c_void_p(256)
    steps = np.array([3, 2], np.uint32)   # not ascending
    cnt = ctypes.c_int64(0)
    rc = lib.gres_compute(fake, 10, 2, 0, steps.ctypes.data_as(ctypes.c_void_p), 2, None,
                          fake, 1 << 30, fake, fake, None, ctypes.byref(cnt), None, None)
    assert rc == 1 and b"ascending" in lib.gres_last_error()
    steps = np.array([0, 2], np.uint32)   # zero width
    rc = lib.gres_compute(fake, 10, 2, 0, steps.ctypes.data_as(ctypes.c_void_p), 2, None,
                          fake, 1 << 30, fake, fake, None, ctypes.byref(cnt), None, None)
    assert rc == 1
    steps = np.array([1, 2], np.uint32)
    rc = lib.gres_compute(fake, 10, 2, 7, steps.ctypes.data_as(ctypes.c_void_p), 2, None,
                          fake, 1 << 30, fake, fake, None, ctypes.byref(cnt), None, None)
    assert rc == 1 and b"dir" in lib.gres_last_error()
    rc = lib.gres_compute(fake, 10, 2, 0, steps.ctypes.data_as(ctypes.c_void_p), 2, None,
                          fake, 16, fake, fake, None, ctypes.byref(cnt), None, None)
    assert rc == 1 and b"workspace" in lib.gres_last_error()
    bad_plan = G.plan(G.PART_SLICED, slice_dim=5)
    rc = lib.gres_compute(fake, 10, 2, 0, steps.ctypes.data_as(ctypes.c_void_p), 2,
                          ctypes.byref(bad_plan), fake, 1 << 30, fake, fake, None,
                          ctypes.byref(cnt), None, None)
    assert rc == 1 and b"slice_dim" in lib.gres_last_error()
    rc = lib.sky_compute(fake, 10, 0, 0, fake, 1 << 30, fake, None, ctypes.byref(cnt), None)
    assert rc == 1


def _apply_magic(v, m, s1, s2):
    v = v.astype(np.uint64)
    t = (np.uint64(m) * v) >> np.uint64(32)
    return ((t + ((v - t) >> np.uint64(s1))) >> np.uint64(s2)).astype(np.uint64)


def test_division_constants_exhaustive_20bit():
    """Granlund-Montgomery constants give floor(v / delta) for every v < 2^20 and every width used."""
    v = np.arange(1 << 20, dtype=np.uint64)
    for delta in sorted(set(steps_log(256, 16).tolist()) | set(steps_linear(64, 64).tolist())):
        m, s1, s2 = G.udiv_magic(delta)
        np.testing.assert_array_equal(_apply_magic(v, m, s1, s2), v // np.uint64(delta))


def test_division_constants_full_range_samples():
    rng = np.random.default_rng(0)
    deltas = np.concatenate([rng.integers(1, 1 << 32, size=300, dtype=np.uint64),
                             [1, 2, 3, 5, 7, (1 << 31) - 1, 1 << 31, (1 << 31) + 1,
                              0xFFFFFFFE, 0xFFFFFFFF]]).astype(np.uint64)
    v = np.concatenate([rng.integers(0, 1 << 32, size=20000, dtype=np.uint64),
                        [0, 1, 0xFFFFFFFF, 0xFFFFFFFE, 1 << 31]]).astype(np.uint64)
    for delta in deltas.tolist():
        m, s1, s2 = G.udiv_magic(delta)
        edges = np.array([x for q in (1, 2, 3) for x in (q * delta - 1, q * delta, q * delta + 1)
                          if 0 <= x <= 0xFFFFFFFF], dtype=np.uint64)
        vv = np.concatenate([v, edges])
        np.testing.assert_array_equal(_apply_magic(vv, m, s1, s2), vv // np.uint64(delta))
    with pytest.raises(G.GresError):
        G.udiv_magic(0)


def test_server_argument_checks_need_no_gpu():
    lib = G.load()
    out = ctypes.c_void_p()
    assert lib.gres_serve_create(1 << 30, None, None) == 1
    bad = G.ServeCfg(0, 99, 0, 0, 0)                      # max_inflight out of range
    assert lib.gres_serve_create(1 << 30, ctypes.byref(bad), ctypes.byref(out)) == 1
    bad = G.ServeCfg(1000, 0, 0, 0, 0)                    # max_batch out of range
    assert lib.gres_serve_create(1 << 30, ctypes.byref(bad), ctypes.byref(out)) == 1
    t = ctypes.c_uint64(0)
    steps = np.array([1, 2], np.uint32)
    assert lib.gres_serve_submit(None, 0, steps.ctypes.data_as(ctypes.c_void_p), 2, ctypes.byref(t)) == 1
    assert lib.gres_serve_poll(None, 1, None, 0, None, None, 0) == 1
    assert lib.gres_serve_destroy(None) == 0


def test_partition_argument_checks_need_no_gpu():
    lib = G.load()
    fake = ctypes.c_void_p(256)
    for d, direction, cfg in [(0, 0, None), (9, 0, None), (2, 5, None),
                              (2, 0, G.PlanCfg(scheme=7)),
                              (3, 0, G.PlanCfg(scheme=G.PART_SLICED, p=4, slice_dim=3)),
                              (3, 0, G.PlanCfg(scheme=G.PART_ANGULAR, m=65))]:
        cfgp = ctypes.byref(cfg) if cfg is not None else None
        rc = lib.gres_partition(fake, 10, d, direction, cfgp, fake, 1 << 30, fake, fake, fake, None)
        assert rc == 1, (d, direction)
    # workspace too small / misaligned
    rc = lib.gres_partition(fake, 10, 2, 0, None, fake, 16, fake, fake, fake, None)
    assert rc == 1 and b"workspace" in lib.gres_last_error()
    rc = lib.gres_partition(fake, 10, 2, 0, None, ctypes.c_void_p(260), 1 << 30, fake, fake, fake, None)
    assert rc == 1


def test_gmode_argument_checks_need_no_gpu():
    lib = G.load()
    fake = ctypes.c_void_p(256)
    cnt = ctypes.c_int64(0)
    for bits, gl in [(0, [4, 2]), (33, [4, 2]), (20, [2, 4]), (20, [3, 3]), (20, [2, 0])]:
        g = np.array(gl, np.uint32)
        rc = lib.gres_compute_g(fake, 10, 2, 0, bits, g.ctypes.data_as(ctypes.c_void_p), len(g), None,
                                fake, 1 << 30, fake, fake, None, ctypes.byref(cnt), None, None)
        assert rc == 1, (bits, gl)


def test_gres_reps_flag_rejected_where_not_supported():
    lib = G.load()
    out = ctypes.c_void_p()
    cfg = G.plan(G.PART_GRID, gres_reps=True)
    data = np.zeros((4, 2), np.uint32)
    rc = lib.gres_dataset_create(data.ctypes.data_as(ctypes.c_void_p), 4, 2, 0, ctypes.byref(cfg), 1, None,
                                 ctypes.byref(out))
    assert rc == 1 and b"flags" in lib.gres_last_error()
    bad = G.PlanCfg(G.PART_GRID, 0, 0, 0, 0, 0, 4, 0)   # an unknown flag bit
    fake = ctypes.c_void_p(256)
    steps = np.array([1, 2], np.uint32)
    cnt = ctypes.c_int64(0)
    rc = lib.gres_compute(fake, 10, 2, 0, steps.ctypes.data_as(ctypes.c_void_p), 2, ctypes.byref(bad),
                          fake, 1 << 30, fake, fake, None, ctypes.byref(cnt), None, None)
    assert rc == 1


def test_test_peak_probe_argument_checks_need_no_gpu():
    lib = G.load()
    fake = ctypes.c_void_p(256)
    ops = ctypes.c_double(0.0)
    for d, iters, blocks, sink, out in [(0, 10, 0, fake, ops), (9, 10, 0, fake, ops), (4, 0, 0, fake, ops),
                                        (4, 10, -1, fake, ops), (4, 10, 0, None, ops)]:
        rc = lib.gres_test_peak_probe(d, iters, blocks, sink, None, ctypes.byref(out) if out is not None else None)
        assert rc == 1, (d, iters, blocks)
    rc = lib.gres_test_peak_probe(4, 10, 0, fake, None, None)
    assert rc == 1 and b"NULL" in lib.gres_last_error()

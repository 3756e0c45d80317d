"""Python access to the plain C oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the package smoke check
and by the benchmark's CPU-baseline leg. The product path (the CUDA library
and its binding) never imports this module, and this module imports nothing
from the product package.

``build()`` compiles ``oracle.c`` with gcc into ``oracle/_build/liboracle.so``
(OpenMP when available). Every wrapper takes and returns numpy arrays.
``GRES_ORACLE_LIB`` names another build of ``oracle.c`` to load instead (the
mutation test uses it to check that the pins reject a planted mistake).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_u32p = ctypes.POINTER(ctypes.c_uint32)


def build(force: bool = False) -> str:
    """Compile the oracle if its shared object is missing or older than the source."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True, text=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True, text=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        override = os.environ.get("GRES_ORACLE_LIB")
        lib = ctypes.CDLL(override if override else build())
        lib.oracle_dominates.restype = ctypes.c_int
        lib.oracle_dominates.argtypes = [_u32p, _u32p, ctypes.c_int, ctypes.c_int]
        for name in ("oracle_skyline_bnl", "oracle_skyline_allpairs"):
            f = getattr(lib, name)
            f.restype = ctypes.c_int64
            f.argtypes = [_u32p, ctypes.c_int64, ctypes.c_int, ctypes.c_int, _i64p]
        lib.oracle_skyline_member.restype = None
        lib.oracle_skyline_member.argtypes = [_u32p, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                              _i64p, ctypes.c_int64, _i32p, ctypes.c_int]
        lib.oracle_gproj.restype = None
        lib.oracle_gproj.argtypes = [_u32p, ctypes.c_int64, ctypes.c_uint32, _u32p]
        lib.oracle_gres.restype = None
        lib.oracle_gres.argtypes = [_u32p, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                    _i64p, ctypes.c_int64, _i64p, ctypes.c_int64,
                                    _u32p, ctypes.c_int32, _i32p, ctypes.c_int]
        lib.oracle_gres_literal.restype = ctypes.c_int
        lib.oracle_gres_literal.argtypes = [_u32p, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                            _i64p, ctypes.c_int64, _u32p, ctypes.c_int32, _i32p]
        lib.oracle_gres_glist.restype = None
        lib.oracle_gres_glist.argtypes = [_u32p, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, _i64p, ctypes.c_int64, _i64p,
                                          ctypes.c_int64, _u32p, ctypes.c_int32, _i32p]
        lib.oracle_min_gap.restype = ctypes.c_uint32
        lib.oracle_min_gap.argtypes = [_u32p, ctypes.c_int64, ctypes.c_int]
        for name in ("oracle_grid_pid", "oracle_angular_pid"):
            f = getattr(lib, name)
            f.restype = None
            f.argtypes = [_u32p, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int, _i64p]
        lib.oracle_cell_grid_dominates.restype = ctypes.c_int
        lib.oracle_cell_grid_dominates.argtypes = [ctypes.c_int64, ctypes.c_int64,
                                                   ctypes.c_int, ctypes.c_int]
        lib.oracle_sliced_pid.restype = None
        lib.oracle_sliced_pid.argtypes = [_u32p, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_int, _i64p]
        lib.oracle_max_threads.restype = ctypes.c_int
        lib.oracle_max_threads.argtypes = []
        _lib = lib
        return lib


def _rows(data) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(data, dtype=np.uint32))
    if a.ndim != 2:
        raise ValueError("data must be 2-D (n, d)")
    return a


def _p(a, t):
    return a.ctypes.data_as(t)


def _dir(direction) -> int:
    if direction in (0, "min", "MIN"):
        return 0
    if direction in (1, "max", "MAX"):
        return 1
    raise ValueError(f"bad direction {direction!r}")


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def dominates(s, t, direction="min") -> bool:
    s = np.ascontiguousarray(np.asarray(s, dtype=np.uint32))
    t = np.ascontiguousarray(np.asarray(t, dtype=np.uint32))
    return bool(_load().oracle_dominates(_p(s, _u32p), _p(t, _u32p), len(s), _dir(direction)))


def skyline_bnl(data, direction="min") -> np.ndarray:
    a = _rows(data)
    out = np.empty(max(len(a), 1), dtype=np.int64)
    c = _load().oracle_skyline_bnl(_p(a, _u32p), len(a), a.shape[1], _dir(direction), _p(out, _i64p))
    return out[:c].copy()


def skyline_allpairs(data, direction="min") -> np.ndarray:
    a = _rows(data)
    out = np.empty(max(len(a), 1), dtype=np.int64)
    c = _load().oracle_skyline_allpairs(_p(a, _u32p), len(a), a.shape[1], _dir(direction),
                                        _p(out, _i64p))
    return out[:c].copy()


def skyline_member(data, rows=None, direction="min", threads=1) -> np.ndarray:
    """Def. 1 row by row: a bool per asked row (default: every row), True iff no row of
    ``data`` dominates it."""
    a = _rows(data)
    rw = _idx(rows, len(a))
    out = np.empty(max(len(rw), 1), dtype=np.int32)
    _load().oracle_skyline_member(_p(a, _u32p), len(a), a.shape[1], _dir(direction),
                                  _p(rw, _i64p), len(rw), _p(out, _i32p), int(threads))
    return out[:len(rw)].astype(bool)


def skyline_threaded(data, direction="min", threads=1) -> np.ndarray:
    """Sky(r) as ascending row numbers: Def. 1 asked for every row, OpenMP over the rows."""
    return np.flatnonzero(skyline_member(data, None, direction, threads)).astype(np.int64)


def gproj(values, delta: int) -> np.ndarray:
    v = np.ascontiguousarray(np.asarray(values, dtype=np.uint32))
    out = np.empty_like(v)
    _load().oracle_gproj(_p(v, _u32p), v.size, int(delta), _p(out, _u32p))
    return out


def _idx(x, n) -> np.ndarray:
    if x is None:
        return np.arange(n, dtype=np.int64)
    return np.ascontiguousarray(np.asarray(x, dtype=np.int64))


def gres(data, steps, direction="min", candidates=None, targets=None, threads=1) -> np.ndarray:
    """First exit step index per target (K = never), candidates default to all rows."""
    a = _rows(data)
    st = np.ascontiguousarray(np.asarray(steps, dtype=np.uint32))
    cand = _idx(candidates, len(a))
    tg = _idx(targets, len(a))
    out = np.empty(max(len(tg), 1), dtype=np.int32)
    _load().oracle_gres(_p(a, _u32p), len(a), a.shape[1], _dir(direction),
                        _p(cand, _i64p), len(cand), _p(tg, _i64p), len(tg),
                        _p(st, _u32p), len(st), _p(out, _i32p), int(threads))
    return out[:len(tg)].copy()


def gres_literal(data, steps, direction="min", targets=None) -> np.ndarray:
    a = _rows(data)
    st = np.ascontiguousarray(np.asarray(steps, dtype=np.uint32))
    tg = _idx(targets, len(a))
    out = np.empty(max(len(tg), 1), dtype=np.int32)
    rc = _load().oracle_gres_literal(_p(a, _u32p), len(a), a.shape[1], _dir(direction),
                                     _p(tg, _i64p), len(tg), _p(st, _u32p), len(st),
                                     _p(out, _i32p))
    if rc != 0:
        raise MemoryError("oracle_gres_literal: allocation failed")
    return out[:len(tg)].copy()


def gres_glist(data, bits: int, glist, direction="min", candidates=None,
               targets=None) -> np.ndarray:
    """First g (in the order of ``glist``) at which each target leaves the skyline, else 1."""
    a = _rows(data)
    cand = _idx(candidates, len(a))
    tg = _idx(targets, len(a))
    gl = np.ascontiguousarray(np.asarray(glist, dtype=np.uint32))
    out = np.empty(max(len(tg), 1), dtype=np.int32)
    _load().oracle_gres_glist(_p(a, _u32p), len(a), a.shape[1], _dir(direction), int(bits),
                              _p(cand, _i64p), len(cand), _p(tg, _i64p), len(tg),
                              _p(gl, _u32p), len(gl), _p(out, _i32p))
    return out[:len(tg)].copy()


def gres_gmode(data, bits: int, g_bar: int, direction="min", candidates=None,
               targets=None) -> np.ndarray:
    """Algorithm 1 with the paper's grid parameter: g = g_bar, g_bar - 1, ..., 2."""
    return gres_glist(data, bits, np.arange(int(g_bar), 1, -1), direction, candidates, targets)


def min_gap(data) -> int:
    a = _rows(data)
    return int(_load().oracle_min_gap(_p(a, _u32p), len(a), a.shape[1]))


def grid_pid(data, m: int, direction="min") -> np.ndarray:
    a = _rows(data)
    out = np.empty(max(len(a), 1), dtype=np.int64)
    _load().oracle_grid_pid(_p(a, _u32p), len(a), a.shape[1], _dir(direction), int(m),
                            _p(out, _i64p))
    return out[:len(a)].copy()


def angular_pid(data, m: int, direction="min") -> np.ndarray:
    a = _rows(data)
    out = np.empty(max(len(a), 1), dtype=np.int64)
    _load().oracle_angular_pid(_p(a, _u32p), len(a), a.shape[1], _dir(direction), int(m),
                               _p(out, _i64p))
    return out[:len(a)].copy()


def sliced_pid(data, p: int, dim: int = 0, direction="min") -> np.ndarray:
    a = _rows(data)
    out = np.empty(max(len(a), 1), dtype=np.int64)
    _load().oracle_sliced_pid(_p(a, _u32p), len(a), a.shape[1], _dir(direction), int(dim),
                              int(p), _p(out, _i64p))
    return out[:len(a)].copy()


def cell_grid_dominates(a: int, b: int, d: int, m: int) -> bool:
    return bool(_load().oracle_cell_grid_dominates(int(a), int(b), int(d), int(m)))


def gres_all(data, steps, direction="min", threads=1):
    """Skyline (BNL) then gres over Sky(r) for every skyline row: (sky_idx, step_idx)."""
    sky = skyline_bnl(data, direction)
    out = gres(data, steps, direction, candidates=sky, targets=sky, threads=threads)
    return sky, out

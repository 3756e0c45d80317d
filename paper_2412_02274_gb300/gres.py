"""Thin Python binding of libgres (include/gres.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of the library. Device buffers are torch tensors (PyTorch provides
device memory and streams); uint32 data travels as int32 tensors of the same
bits. There is no CPU fallback: if the library cannot be built or loaded, or
no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

from . import build as _build

MIN, MAX = 0, 1
PART_NONE, PART_GRID, PART_ANGULAR, PART_SLICED = 0, 1, 2, 3
FLAG_COUNT_TESTS = 1
FLAG_GRES_REPS = 2
FLAG_COUNT_PARTS = 4

_STATUS = {0: "GRES_OK", 1: "GRES_EINVAL", 2: "GRES_ENOMEM", 3: "GRES_EAGAIN",
           4: "GRES_ETIMEOUT", 5: "GRES_ECUDA", 6: "GRES_EINTERNAL"}

_lock = threading.Lock()
_lib = None

_p = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_u32 = ctypes.c_uint32
_size = ctypes.c_size_t


class GresError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class PlanCfg(ctypes.Structure):
    """``gres_plan_cfg``: candidate grouping and kernel shape (speed only)."""
    _fields_ = [("scheme", _i32), ("m", _i32), ("p", _i32), ("slice_dim", _i32),
                ("reps", _i32), ("slots", _i32), ("flags", _i32), ("reserved", _i32)]


class ServeCfg(ctypes.Structure):
    """``gres_serve_cfg``."""
    _fields_ = [("max_batch", _i32), ("max_inflight", _i32), ("queue_capacity", _i32), ("max_k", _i32),
                ("start_paused", _i32), ("chunk_targets", _i32)]


class Instance(ctypes.Structure):
    """``gres_instance``: one problem of a gres_batch call (device pointers)."""
    _fields_ = [("d_data", _p), ("n", _i64), ("d", _i32), ("dir", _i32), ("d_steps", _p),
                ("k", _i32), ("cfg", PlanCfg), ("d_sky_idx", _p), ("d_step_idx", _p),
                ("d_sky_count", _p)]


def plan(scheme: int = PART_GRID, m: int = 0, p: int = 0, slice_dim: int = 0, reps: int = 0,
         slots: int = 0, count_tests: bool = False, gres_reps: bool = False,
         count_parts: bool = False) -> PlanCfg:
    flags = ((FLAG_COUNT_TESTS if count_tests or count_parts else 0) | (FLAG_GRES_REPS if gres_reps else 0)
             | (FLAG_COUNT_PARTS if count_parts else 0))
    return PlanCfg(scheme, m, p, slice_dim, reps, slots, flags, 0)


def plan_partitions(cfg: PlanCfg | None, d: int) -> int:
    """Partitions P of a plan for d attributes (the per-partition counts of count_parts
    need a tests tensor of 2 + 4 P int64)."""
    out = _i64(0)
    _check(load().gres_plan_partitions(ctypes.byref(cfg) if cfg is not None else None, int(d),
                                       ctypes.byref(out)))
    return int(out.value)


def library_path() -> str:
    return _build.LIB


def load():
    """Build (if needed) and load libgres; raise if that is impossible."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build()
        lib = ctypes.CDLL(path)
        lib.gres_last_error.restype = ctypes.c_char_p
        lib.gres_version.restype = ctypes.c_char_p
        lib.gres_workspace_size.argtypes = [_i64, _i32, _i32, ctypes.POINTER(_size)]
        lib.gres_workspace_size_host.argtypes = [_i64, _i32, _i32, ctypes.POINTER(_size)]
        lib.sky_compute.argtypes = [_p, _i64, _i32, _i32, _p, _size, _p, _p, _p, _p]
        lib.gres_compute.argtypes = [_p, _i64, _i32, _i32, _p, _i32, ctypes.POINTER(PlanCfg),
                                     _p, _size, _p, _p, _p, _p, _p, _p]
        lib.gres_compute_host.argtypes = [_p, _i64, _i32, _i32, _p, _i32, ctypes.POINTER(PlanCfg),
                                          _p, _size, _p, _p, _p, _p]
        lib.gres_gproj.argtypes = [_p, _i64, _p, _i32, _p, _p]
        lib.gres_compute_g.argtypes = [_p, _i64, _i32, _i32, _i32, _p, _i32, ctypes.POINTER(PlanCfg),
                                       _p, _size, _p, _p, _p, _p, _p, _p]
        lib.gres_partition.argtypes = [_p, _i64, _i32, _i32, ctypes.POINTER(PlanCfg), _p, _size,
                                       _p, _p, _p, _p]
        lib.gres_udiv_magic.argtypes = [_u32, ctypes.POINTER(_u32), ctypes.POINTER(_u32),
                                        ctypes.POINTER(_u32)]
        lib.gres_barrier_probe.argtypes = [_i32, _p, _p, ctypes.POINTER(_u32)]
        lib.gres_plan_partitions.argtypes = [ctypes.POINTER(PlanCfg), _i32, ctypes.POINTER(_i64)]
        lib.gres_test_peak_probe.argtypes = [_i32, _i32, _i32, _p, _p, ctypes.POINTER(ctypes.c_double)]
        lib.gres_launch_count.restype = ctypes.c_ulonglong
        lib.gres_launch_count.argtypes = []
        lib.gres_timing_enable.argtypes = [_i32]
        lib.gres_timing_read.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_i64), _i32]
        lib.gres_dataset_create.argtypes = [_p, _i64, _i32, _i32, ctypes.POINTER(PlanCfg), _i32, _p,
                                            ctypes.POINTER(_p)]
        lib.gres_dataset_destroy.argtypes = [_p]
        lib.gres_dataset_info.argtypes = [_p, ctypes.POINTER(_i64), ctypes.POINTER(_i32),
                                          ctypes.POINTER(_i64), ctypes.POINTER(_size)]
        lib.gres_dataset_sky_idx.argtypes = [_p, _p, _i32, _p]
        lib.gres_query_workspace_size.argtypes = [_i32, ctypes.POINTER(_size)]
        lib.gres_query.argtypes = [_p, _p, _i32, _p, _size, _p, _p]
        lib.gres_batch_workspace_size.argtypes = [ctypes.POINTER(Instance), _i32, ctypes.POINTER(_size)]
        lib.gres_batch.argtypes = [ctypes.POINTER(Instance), _i32, _p, _size, _p]
        lib.gres_serve_create.argtypes = [_size, ctypes.POINTER(ServeCfg), ctypes.POINTER(_p)]
        lib.gres_serve_add_dataset.argtypes = [_p, _p, _i64, _i32, _i32, ctypes.POINTER(PlanCfg), _i32,
                                               ctypes.POINTER(_i32)]
        lib.gres_serve_remove_dataset.argtypes = [_p, _i32]
        lib.gres_serve_submit.argtypes = [_p, _i32, _p, _i32, ctypes.POINTER(ctypes.c_uint64)]
        lib.gres_serve_poll.argtypes = [_p, ctypes.c_uint64, _p, _i64, ctypes.POINTER(_i64),
                                        ctypes.POINTER(_i64), _i64]
        lib.gres_serve_sky_idx.argtypes = [_p, _i32, _p, _i64, ctypes.POINTER(_i64)]
        lib.gres_serve_cancel.argtypes = [_p, ctypes.c_uint64]
        lib.gres_serve_resume.argtypes = [_p]
        lib.gres_serve_pause.argtypes = [_p]
        lib.gres_serve_stats.argtypes = [_p, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                                         ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(_size)]
        lib.gres_serve_destroy.argtypes = [_p]
        for name in ("gres_serve_create", "gres_serve_add_dataset", "gres_serve_remove_dataset",
                     "gres_serve_submit", "gres_serve_poll", "gres_serve_sky_idx", "gres_serve_cancel",
                     "gres_serve_resume",
                     "gres_serve_pause", "gres_serve_stats", "gres_serve_destroy"):
            getattr(lib, name).restype = ctypes.c_int
        for name in ("gres_workspace_size", "gres_workspace_size_host", "sky_compute",
                     "gres_compute", "gres_compute_host", "gres_gproj", "gres_udiv_magic",
                     "gres_timing_enable", "gres_timing_read", "gres_dataset_create",
                     "gres_dataset_destroy", "gres_dataset_info", "gres_dataset_sky_idx",
                     "gres_query_workspace_size", "gres_query", "gres_batch_workspace_size",
                     "gres_batch", "gres_test_peak_probe", "gres_barrier_probe", "gres_plan_partitions"):
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib


def _check(status: int):
    if status != 0:
        raise GresError(status, load().gres_last_error().decode())


def version() -> str:
    return load().gres_version().decode()


def workspace_size(n: int, d: int, k: int = 1, host: bool = False) -> int:
    out = _size(0)
    fn = load().gres_workspace_size_host if host else load().gres_workspace_size
    _check(fn(int(n), int(d), int(k), ctypes.byref(out)))
    return int(out.value)


STAGES = ("skyline", "partition", "dominance")


def launch_count() -> int:
    """Kernels queued by libgres since it was loaded."""
    return int(load().gres_launch_count())


def timing_enable(on: bool = True) -> None:
    _check(load().gres_timing_enable(1 if on else 0))


def timing_read() -> dict:
    """{stage: (summed ms, intervals)} for the events recorded since the last read."""
    ms = (ctypes.c_double * len(STAGES))()
    n = (_i64 * len(STAGES))()
    _check(load().gres_timing_read(ms, n, len(STAGES)))
    return {name: (float(ms[i]), int(n[i])) for i, name in enumerate(STAGES)}


def udiv_magic(delta: int):
    m, s1, s2 = _u32(0), _u32(0), _u32(0)
    _check(load().gres_udiv_magic(int(delta), ctypes.byref(m), ctypes.byref(s1), ctypes.byref(s2)))
    return int(m.value), int(s1.value), int(s2.value)


def test_peak_probe(d: int, iters: int, sink, blocks: int = 0, stream=None) -> float:
    """Queue the dominance-test peak probe on ``stream``; returns the compare lane-ops of the
    launch (time it with CUDA events on that stream). ``sink``: a CUDA tensor of >= 8 bytes."""
    ops = ctypes.c_double(0.0)
    _check(load().gres_test_peak_probe(int(d), int(iters), int(blocks), _ptr(sink), _stream_ptr(stream),
                                       ctypes.byref(ops)))
    return float(ops.value)


def barrier_probe(absent: int, stream=None) -> tuple[int, int]:
    """Runs the bounded grid-wide wait check (gres_barrier_probe): (status code, status word)."""
    torch = _torch()
    words = torch.zeros(4, dtype=torch.int32, device="cuda")
    st = _u32(0)
    rc = load().gres_barrier_probe(int(absent), _ptr(words), _stream_ptr(stream), ctypes.byref(st))
    return int(rc), int(st.value)


# ---- torch-side helpers (device memory and streams) ---------------------------

def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libgres needs a CUDA GPU; none is available")
    return torch


def to_device_u32(a, device="cuda"):
    """numpy uint32 array -> contiguous int32 CUDA tensor holding the same bits."""
    torch = _torch()
    a = np.ascontiguousarray(np.asarray(a, dtype=np.uint32))
    return torch.from_numpy(a.view(np.int32)).to(device)


def _stream_ptr(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _steps_array(steps) -> np.ndarray:
    st = np.ascontiguousarray(np.asarray(steps, dtype=np.uint64))
    if st.ndim != 1 or (st.size and (st.min() < 1 or st.max() > 0xFFFFFFFF)):
        raise ValueError("steps must be a 1-D list of widths in [1, 2^32)")
    return st.astype(np.uint32)


@dataclass
class Workspace:
    tensor: object
    nbytes: int


def alloc_workspace(n: int, d: int, k: int = 1, host: bool = False) -> Workspace:
    torch = _torch()
    nbytes = workspace_size(n, d, k, host)
    return Workspace(torch.empty(nbytes, dtype=torch.uint8, device="cuda"), nbytes)


def sky_compute(data, direction: int = MIN, ws: Workspace | None = None, stream=None):
    """Skyline row numbers (ascending int64 CUDA tensor) of an (n, d) int32/uint32 CUDA tensor."""
    torch = _torch()
    n, d = int(data.shape[0]), int(data.shape[1])
    ws = ws or alloc_workspace(n, d, 1)
    sky = torch.empty(max(n, 1), dtype=torch.int64, device=data.device)
    cnt = ctypes.c_int64(0)
    _check(load().sky_compute(_ptr(data), n, d, int(direction), _ptr(ws.tensor), ws.nbytes,
                              _ptr(sky), None, ctypes.byref(cnt), _stream_ptr(stream)))
    return sky[: cnt.value]


def gres_compute(data, steps, direction: int = MIN, cfg: PlanCfg | None = None,
                 ws: Workspace | None = None, stream=None, sync: bool = True,
                 out=None, tests=None):
    """Skyline and per-tuple first exit step.

    ``data``: (n, d) int32 CUDA tensor (uint32 bits). Returns
    ``(sky_idx[S], step_idx[S])`` CUDA tensors when ``sync`` (one host wait
    for S); otherwise queues everything and returns ``(sky_idx, step_idx,
    d_count)`` full-capacity tensors with S on the device (graph-capturable).
    """
    torch = _torch()
    n, d = int(data.shape[0]), int(data.shape[1])
    st = _steps_array(steps)
    k = len(st)
    ws = ws or alloc_workspace(n, d, k)
    if out is None:
        sky = torch.empty(max(n, 1), dtype=torch.int64, device=data.device)
        res = torch.empty(max(n, 1), dtype=torch.int32, device=data.device)
        dcnt = torch.zeros(1, dtype=torch.int64, device=data.device)
    else:
        sky, res, dcnt = out
    cfgp = ctypes.byref(cfg) if cfg is not None else None
    cnt = ctypes.c_int64(0)
    _check(load().gres_compute(_ptr(data), n, d, int(direction),
                               st.ctypes.data_as(ctypes.c_void_p), k, cfgp,
                               _ptr(ws.tensor), ws.nbytes, _ptr(sky), _ptr(res), _ptr(dcnt),
                               ctypes.byref(cnt) if sync else None, _ptr(tests),
                               _stream_ptr(stream)))
    if sync:
        return sky[: cnt.value], res[: cnt.value]
    return sky, res, dcnt


def gres_compute_g(data, bits: int, g_list, direction: int = MIN, cfg: PlanCfg | None = None,
                   ws: Workspace | None = None, stream=None, tests=None):
    """The paper's grid-parameter form: projection floor(v g / 2^bits) for each g of
    ``g_list`` (strictly descending). Returns ``(sky_idx[S], idx[S])`` CUDA tensors, idx
    the first position in ``g_list`` at which the tuple leaves the skyline, len(g_list)
    if never (the paper's gres = 1)."""
    torch = _torch()
    n, d = int(data.shape[0]), int(data.shape[1])
    gl = _steps_array(g_list)
    k = len(gl)
    ws = ws or alloc_workspace(n, d, k)
    sky = torch.empty(max(n, 1), dtype=torch.int64, device=data.device)
    res = torch.empty(max(n, 1), dtype=torch.int32, device=data.device)
    cfgp = ctypes.byref(cfg) if cfg is not None else None
    cnt = ctypes.c_int64(0)
    _check(load().gres_compute_g(_ptr(data), n, d, int(direction), int(bits),
                                 gl.ctypes.data_as(ctypes.c_void_p), k, cfgp,
                                 _ptr(ws.tensor), ws.nbytes, _ptr(sky), _ptr(res), None,
                                 ctypes.byref(cnt), _ptr(tests), _stream_ptr(stream)))
    return sky[: cnt.value], res[: cnt.value]


def gres_compute_host(data_host, steps, direction: int = MIN, cfg: PlanCfg | None = None,
                      ws: Workspace | None = None, stream=None, out=None):
    """Host-buffer form: numpy (or pinned torch CPU) uint32 (n, d) in, numpy results out."""
    torch = _torch()
    if isinstance(data_host, np.ndarray):
        a = np.ascontiguousarray(data_host, dtype=np.uint32)
        n, d = a.shape
        ptr = a.ctypes.data_as(ctypes.c_void_p)
    else:
        a = data_host
        n, d = int(a.shape[0]), int(a.shape[1])
        ptr = ctypes.c_void_p(a.data_ptr())
    st = _steps_array(steps)
    k = len(st)
    ws = ws or alloc_workspace(n, d, k, host=True)
    if out is None:
        sky = np.empty(max(n, 1), dtype=np.int64)
        res = np.empty(max(n, 1), dtype=np.int32)
        sky_p, res_p = sky.ctypes.data_as(ctypes.c_void_p), res.ctypes.data_as(ctypes.c_void_p)
    else:
        sky, res = out
        sky_p, res_p = ctypes.c_void_p(sky.data_ptr()), ctypes.c_void_p(res.data_ptr())
    cfgp = ctypes.byref(cfg) if cfg is not None else None
    cnt = ctypes.c_int64(0)
    _check(load().gres_compute_host(ptr, int(n), int(d), int(direction),
                                    st.ctypes.data_as(ctypes.c_void_p), k, cfgp,
                                    _ptr(ws.tensor), ws.nbytes, sky_p, res_p, ctypes.byref(cnt),
                                    _stream_ptr(stream)))
    return sky[: cnt.value], res[: cnt.value]


def gproj(values, steps, stream=None):
    """floor(values / steps[j]) for every width: a (k, count) int32 CUDA tensor (uint32 bits)."""
    torch = _torch()
    st = _steps_array(steps)
    v = values if hasattr(values, "data_ptr") else to_device_u32(values)
    count = int(v.numel())
    out = torch.empty((len(st), max(count, 1)), dtype=torch.int32, device=v.device)
    _check(load().gres_gproj(_ptr(v), count, st.ctypes.data_as(ctypes.c_void_p), len(st),
                             _ptr(out), _stream_ptr(stream)))
    return out[:, :count]


def partition(rows, direction: int = MIN, cfg: PlanCfg | None = None, stream=None):
    """Partition numbers, tile order and tile minima of a candidate set (Sec. 3.1).

    rows: (n, d) uint32 CUDA tensor (int32 bits) or numpy array. Returns CUDA
    tensors (part int64 [n], order int32 [n] (uint32 bits), tile_min int32
    [ceil(n/32), d] (uint32 bits)) once queued on the stream."""
    torch = _torch()
    r = rows if hasattr(rows, "data_ptr") else to_device_u32(rows)
    n, d = int(r.shape[0]), int(r.shape[1])
    dev = r.device
    ws = alloc_workspace(n, d, 1)
    part = torch.empty(max(n, 1), dtype=torch.int64, device=dev)
    order = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    tiles = (n + 31) // 32
    tmin = torch.empty((max(tiles, 1), d), dtype=torch.int32, device=dev)
    cfgp = ctypes.byref(cfg) if cfg is not None else None
    _check(load().gres_partition(_ptr(r), n, d, int(direction), cfgp, _ptr(ws.tensor), ws.nbytes,
                                 _ptr(part), _ptr(order), _ptr(tmin), _stream_ptr(stream)))
    return part[:n], order[:n], tmin[:tiles]


# ---- resident datasets and queries ---------------------------------------------------

class Dataset:
    """A prepared dataset (skyline + candidate tiles on the device) for repeated queries."""

    def __init__(self, data, direction: int = MIN, cfg: PlanCfg | None = None, stream=None):
        import torch
        self._lib = load()
        h = _p()
        cfgp = ctypes.byref(cfg) if cfg is not None else None
        if isinstance(data, np.ndarray):
            a = np.ascontiguousarray(data, dtype=np.uint32)
            n, d = a.shape
            ptr, on_host = a.ctypes.data_as(ctypes.c_void_p), 1
        else:
            a = data
            n, d = int(a.shape[0]), int(a.shape[1])
            ptr, on_host = _ptr(a), 0 if a.is_cuda else 1
        _check(self._lib.gres_dataset_create(ptr, int(n), int(d), int(direction), cfgp, on_host,
                                             _stream_ptr(stream), ctypes.byref(h)))
        self._h = h
        nn, dd, ss, bb = _i64(0), _i32(0), _i64(0), _size(0)
        _check(self._lib.gres_dataset_info(h, ctypes.byref(nn), ctypes.byref(dd), ctypes.byref(ss),
                                           ctypes.byref(bb)))
        self.n, self.d, self.S, self.device_bytes = nn.value, dd.value, ss.value, bb.value
        self._torch = torch

    def sky_idx(self, stream=None):
        out = np.empty(max(self.S, 1), dtype=np.int64)
        _check(self._lib.gres_dataset_sky_idx(self._h, out.ctypes.data_as(ctypes.c_void_p), 1,
                                              _stream_ptr(stream)))
        return out[: self.S]

    def query(self, steps, out=None, qws=None, stream=None):
        """Step index per skyline row (CUDA int32 tensor of S entries), queued on `stream`."""
        torch = self._torch
        st = _steps_array(steps)
        k = len(st)
        if qws is None:
            sz = _size(0)
            _check(self._lib.gres_query_workspace_size(k, ctypes.byref(sz)))
            qws = torch.empty(int(sz.value), dtype=torch.uint8, device="cuda")
        if out is None:
            out = torch.empty(max(self.S, 1), dtype=torch.int32, device="cuda")
        _check(self._lib.gres_query(self._h, st.ctypes.data_as(ctypes.c_void_p), k, _ptr(qws),
                                    qws.numel(), _ptr(out), _stream_ptr(stream)))
        return out[: self.S]

    def close(self):
        if getattr(self, "_h", None):
            _check(self._lib.gres_dataset_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch(problems, stream=None, ws=None):
    """Many gres_compute problems in one gres_batch call.

    ``problems``: list of dicts with ``data`` ((n, d) int32 CUDA tensor), ``steps``
    (1-D int32 CUDA tensor of widths), optional ``direction`` and ``cfg``. Returns the
    per-instance output tensors ``(sky_idx, step_idx, sky_count)`` (full capacity, with
    S on the device) and the ctypes instance array (keep both alive while replaying a
    captured graph)."""
    torch = _torch()
    insts = (Instance * max(len(problems), 1))()
    outs = []
    for i, pr in enumerate(problems):
        x = pr["data"]
        n, d = int(x.shape[0]), int(x.shape[1])
        st = pr["steps"]
        sky = torch.empty(max(n, 1), dtype=torch.int64, device=x.device)
        res = torch.empty(max(n, 1), dtype=torch.int32, device=x.device)
        cnt = torch.zeros(1, dtype=torch.int64, device=x.device)
        cfg = pr.get("cfg") or PlanCfg()
        insts[i] = Instance(x.data_ptr(), n, d, int(pr.get("direction", MIN)), st.data_ptr(), int(st.numel()),
                            cfg, sky.data_ptr(), res.data_ptr(), cnt.data_ptr())
        outs.append((sky, res, cnt))
    if ws is None:
        sz = _size(0)
        _check(load().gres_batch_workspace_size(insts, len(problems), ctypes.byref(sz)))
        ws = torch.empty(int(sz.value), dtype=torch.uint8, device="cuda")
    _check(load().gres_batch(insts, len(problems), _ptr(ws), ws.numel(), _stream_ptr(stream)))
    return outs, insts, ws


# ---- serving --------------------------------------------------------------------------

class Server:
    """A gres query server (resident datasets, continuous batching) on the current GPU."""

    def __init__(self, hbm_budget_bytes: int, max_batch: int = 0, max_inflight: int = 0,
                 queue_capacity: int = 0, max_k: int = 0, start_paused: bool = False,
                 chunk_targets: int = 0):
        _torch()
        self._lib = load()
        h = _p()
        cfg = ServeCfg(max_batch, max_inflight, queue_capacity, max_k, 1 if start_paused else 0,
                       chunk_targets)
        _check(self._lib.gres_serve_create(int(hbm_budget_bytes), ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self.S = {}

    def add_dataset(self, data, direction: int = MIN, cfg: PlanCfg | None = None) -> int:
        a = np.ascontiguousarray(np.asarray(data, dtype=np.uint32))
        n, d = a.shape
        out = _i32(0)
        cfgp = ctypes.byref(cfg) if cfg is not None else None
        _check(self._lib.gres_serve_add_dataset(self._h, a.ctypes.data_as(ctypes.c_void_p), int(n), int(d),
                                                int(direction), cfgp, 1, ctypes.byref(out)))
        return int(out.value)

    def remove_dataset(self, dataset_id: int) -> None:
        _check(self._lib.gres_serve_remove_dataset(self._h, int(dataset_id)))

    def submit(self, dataset_id: int, steps) -> int:
        st = _steps_array(steps)
        t = ctypes.c_uint64(0)
        _check(self._lib.gres_serve_submit(self._h, int(dataset_id), st.ctypes.data_as(ctypes.c_void_p),
                                           len(st), ctypes.byref(t)))
        return int(t.value)

    def poll(self, ticket: int, timeout_us: int = -1, cap: int = 1 << 22):
        """(step_idx numpy int32, latency_ns), or None if not finished within the timeout."""
        out = np.empty(cap, dtype=np.int32)
        S, lat = _i64(0), _i64(0)
        rc = self._lib.gres_serve_poll(self._h, ctypes.c_uint64(ticket), out.ctypes.data_as(ctypes.c_void_p),
                                       cap, ctypes.byref(S), ctypes.byref(lat), int(timeout_us))
        if rc == 3:
            return None
        _check(rc)
        return out[: S.value].copy(), int(lat.value)

    def sky_idx(self, dataset_id: int) -> np.ndarray:
        """The dataset's skyline row numbers (ascending): the rows of every poll result."""
        S = _i64(-1)
        # a first call with no buffer reports S (and GRES_EINVAL when S > 0)
        rc = self._lib.gres_serve_sky_idx(self._h, int(dataset_id), None, 0, ctypes.byref(S))
        if S.value < 0:
            _check(rc)
        out = np.empty(max(S.value, 1), dtype=np.int64)
        _check(self._lib.gres_serve_sky_idx(self._h, int(dataset_id), out.ctypes.data_as(ctypes.c_void_p),
                                            len(out), ctypes.byref(S)))
        return out[: S.value]

    def cancel(self, ticket: int) -> None:
        _check(self._lib.gres_serve_cancel(self._h, ctypes.c_uint64(ticket)))

    def resume(self) -> None:
        _check(self._lib.gres_serve_resume(self._h))

    def pause(self) -> None:
        _check(self._lib.gres_serve_pause(self._h))

    def stats(self) -> dict:
        b, q, l, m = ctypes.c_uint64(0), ctypes.c_uint64(0), ctypes.c_uint64(0), _size(0)
        _check(self._lib.gres_serve_stats(self._h, ctypes.byref(b), ctypes.byref(q), ctypes.byref(l),
                                          ctypes.byref(m)))
        return {"batches": b.value, "queries": q.value, "launches": l.value, "device_bytes": m.value}

    def close(self) -> None:
        if getattr(self, "_h", None):
            _check(self._lib.gres_serve_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

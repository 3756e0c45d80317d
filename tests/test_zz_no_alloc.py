"""gres_compute_static: the entry point for callers that cannot allocate.

Some callers have no way to hand the library a device workspace: for example
a plugin running on another framework's stream whose allocator owns the free
memory, or a latency-critical loop that must not call cudaMalloc (which can
synchronise the device). gres_compute_static serves them from a fixed scratch
array inside the library. This test calls it through the C ABI twice in a row
(on two different datasets, so the second call starts from the first call's
leftovers) and checks both results against gres_compute with a workspace,
exactly. It also checks that sizes beyond the static scratch are refused
before anything is launched. Kept in its own file, collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_2412_02274_gb300 import gres as G
from paper_2412_02274_gb300.inputs import make_dataset, steps_log

pytestmark = pytest.mark.gpu


def _static_entry():
    lib = G.load()
    f = lib.gres_compute_static
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                  ctypes.c_int32, ctypes.POINTER(G.PlanCfg), ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.gres_static_scratch_bytes.restype = ctypes.c_size_t
    return lib, f


def _call_static(f, x, steps, cfg):
    import torch
    n, d = x.shape
    sky = torch.full((n,), -1, dtype=torch.int64, device="cuda")
    res = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    cnt = ctypes.c_int64(-1)
    st = np.ascontiguousarray(steps, dtype=np.uint32)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = f(ctypes.c_void_p(x.data_ptr()), n, d, G.MIN, st.ctypes.data_as(ctypes.c_void_p), len(st),
           ctypes.byref(cfg), ctypes.c_void_p(sky.data_ptr()), ctypes.c_void_p(res.data_ptr()), None,
           ctypes.byref(cnt), stream)
    return rc, sky[: max(cnt.value, 0)].cpu().numpy(), res[: max(cnt.value, 0)].cpu().numpy()


def test_static_scratch_entry_matches_workspace_entry_twice():
    lib, f = _static_entry()
    steps = steps_log(256, 16)
    cfg = G.plan(G.PART_GRID, m=4)
    for dist, n, seed in (("ant", 60000, 3), ("clu", 20000, 4)):
        data = make_dataset(dist, n, 4, bits=20, seed=seed)
        x = G.to_device_u32(data)
        ref_sky, ref_res = G.gres_compute(x, steps, G.MIN, cfg)
        rc, sky, res = _call_static(f, x, steps, cfg)
        assert rc == 0, lib.gres_last_error()
        np.testing.assert_array_equal(sky, ref_sky.cpu().numpy())
        np.testing.assert_array_equal(res, ref_res.cpu().numpy())


def test_static_scratch_entry_allocates_nothing():
    """After a warm-up call, more calls leave the device's free memory unchanged: nothing
    is allocated (outputs are allocated once, up front)."""
    import torch
    lib, f = _static_entry()
    steps = steps_log(256, 16)
    cfg = G.plan(G.PART_GRID, m=4)
    data = make_dataset("ant", 50000, 4, bits=20, seed=8)
    x = G.to_device_u32(data)
    n, d = x.shape
    sky = torch.empty(n, dtype=torch.int64, device="cuda")
    res = torch.empty(n, dtype=torch.int32, device="cuda")
    st = np.ascontiguousarray(steps, dtype=np.uint32)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    cnt = ctypes.c_int64(-1)

    def call():
        return f(ctypes.c_void_p(x.data_ptr()), n, d, G.MIN, st.ctypes.data_as(ctypes.c_void_p), len(st),
                 ctypes.byref(cfg), ctypes.c_void_p(sky.data_ptr()), ctypes.c_void_p(res.data_ptr()), None,
                 ctypes.byref(cnt), stream)

    assert call() == 0, lib.gres_last_error()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(4):
        assert call() == 0, lib.gres_last_error()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_static_scratch_first_call_inside_a_capture_is_refused():
    """A fresh process whose first call of the entry point is inside a stream capture gets
    GRES_EINVAL (the scratch address is looked up outside captures only); after a call
    outside the capture, calls inside one are accepted."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = r"""
import ctypes, sys, numpy as np, torch
sys.path.insert(0, %r)
sys.path.insert(0, %r)
from paper_2412_02274_gb300 import gres as G
from paper_2412_02274_gb300.inputs import make_dataset, steps_log
from test_zz_no_alloc import _static_entry, _call_static
lib, f = _static_entry()
n, d = 5000, 3
x = G.to_device_u32(make_dataset("uni", n, d, bits=20, seed=1))
cfg = G.plan(G.PART_GRID)
st = np.ascontiguousarray(steps_log(64, 16), dtype=np.uint32)
sky = torch.empty(n, dtype=torch.int64, device="cuda")
res = torch.empty(n, dtype=torch.int32, device="cuda")
s = torch.cuda.Stream()
s.wait_stream(torch.cuda.current_stream())
torch.cuda.synchronize()
g = torch.cuda.CUDAGraph()
with torch.cuda.graph(g, stream=s, capture_error_mode="relaxed"):
    rc = f(ctypes.c_void_p(x.data_ptr()), n, d, G.MIN, st.ctypes.data_as(ctypes.c_void_p), len(st),
           ctypes.byref(cfg), ctypes.c_void_p(sky.data_ptr()), ctypes.c_void_p(res.data_ptr()), None,
           None, ctypes.c_void_p(s.cuda_stream))
print("RC", rc, lib.gres_last_error().decode())
rc2, sky2, res2 = _call_static(f, x, st, cfg)
ref_sky, ref_res = G.gres_compute(x, st, G.MIN, cfg)
print("RC2", rc2, bool(np.array_equal(res2, ref_res.cpu().numpy())))
""" % (root, os.path.join(root, "tests"))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600, cwd=root)
    assert out.returncode == 0, out.stderr[-3000:]
    lines = dict(l.split(" ", 1) for l in out.stdout.splitlines() if l.startswith("RC"))
    assert lines["RC"].startswith("1 ") and "before any stream capture" in lines["RC"]
    assert lines["RC2"] == "0 True"


def test_static_scratch_refuses_sizes_beyond_its_limit():
    import torch
    lib, f = _static_entry()
    limit = int(lib.gres_static_scratch_bytes())
    assert limit == 16 << 20
    n, d = 2_000_000, 4
    assert G.workspace_size(n, d, 256) > limit
    x = torch.empty((1, d), dtype=torch.int32, device="cuda")   # never read: refused first
    rc, _, _ = _call_static(f, x.expand(n, d), steps_log(256, 16), G.plan(G.PART_GRID))
    assert rc == 1 and b"static scratch" in lib.gres_last_error()

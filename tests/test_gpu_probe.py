"""The dominance-test peak probe (the roofline denominator of the grid-dominance kernel)."""
import pytest

from paper_2412_02274_gb300 import gres as G

pytestmark = pytest.mark.gpu


def test_probe_counts_and_runs():
    import torch
    sink = torch.zeros(1, dtype=torch.int64, device="cuda")
    for d in (1, 4, 8):
        ops = G.test_peak_probe(d, 64, sink, blocks=152)
        assert ops == 152 * 256 * 64 * 16 * 2 * d
        full = G.test_peak_probe(d, 16, sink)   # one full wave: a whole number of SMs' worth
        assert full > 0 and full % (256 * 16 * 16 * 2 * d) == 0
    torch.cuda.synchronize()
    assert int(sink.item()) == 0   # the sink is written only on an impossible count


def test_grid_barrier_wait_is_bounded():
    """The cooperative sorts' grid-wide barrier gives up after a bounded wait: with one
    block kept away on purpose the others flag the timeout and return (GRES_ETIMEOUT,
    no fault), and the context keeps working afterwards."""
    import time
    import numpy as np
    from paper_2412_02274_gb300.inputs import make_dataset, steps_log
    rc, status = G.barrier_probe(-1)
    assert (rc, status) == (0, 0)
    t0 = time.perf_counter()
    rc, status = G.barrier_probe(3)
    assert time.perf_counter() - t0 < 30.0
    assert rc == 4 and status & 1          # GRES_ETIMEOUT, timeout bit
    rc, status = G.barrier_probe(-1)
    assert (rc, status) == (0, 0)
    data = make_dataset("ant", 2000, 3, bits=16, seed=3)
    sky, res = G.gres_compute(G.to_device_u32(data), steps_log(32, 14))
    assert len(sky) > 0 and int(res.max().item()) <= 32

"""GPU: the query server -- continuous batching over resident datasets.

Results must be identical alone and in the mix (bit-exact: every result is an
integer and each target is computed independently of the others). Failure
paths are made on the host: a full queue, a wait that runs out, a cancelled
query, an HBM budget that is too small.
"""
import time

import numpy as np
import pytest

from paper_2412_02274_gb300 import gres as G
from paper_2412_02274_gb300.inputs import make_dataset, steps_log

pytestmark = pytest.mark.gpu

EINVAL, ENOMEM, EAGAIN = 1, 2, 3


def _datasets():
    specs = [("ant", 20000, 4, G.MIN, G.plan(G.PART_GRID, m=4)),
             ("uni", 60000, 6, G.MIN, G.plan(G.PART_ANGULAR, m=2)),
             ("clu", 30000, 3, G.MAX, G.plan(G.PART_SLICED, p=32)),
             ("ant", 5000, 8, G.MIN, G.plan(G.PART_GRID, slots=4)),
             ("uni", 2000, 2, G.MAX, G.plan(G.PART_NONE)),
             ("ant", 40000, 5, G.MIN, G.plan(G.PART_SLICED, p=64))]
    return [(make_dataset(dist, n, d, bits=20, seed=10 + i), direction, cfg)
            for i, (dist, n, d, direction, cfg) in enumerate(specs)]


def test_results_alone_and_in_the_mix():
    rng = np.random.default_rng(3)
    dsets = _datasets()
    sv = G.Server(8 << 30, max_batch=48, max_inflight=3)
    ids = [sv.add_dataset(data, direction, cfg) for data, direction, cfg in dsets]
    alone = [G.Dataset(data, direction, cfg) for data, direction, cfg in dsets]
    queries = [(int(rng.integers(0, len(ids))), steps_log(int(rng.integers(64, 257)), 16)) for _ in range(200)]
    tickets = [sv.submit(ids[j], steps) for j, steps in queries]
    for t, (j, steps) in zip(tickets, queries):
        got, lat = sv.poll(t)
        assert lat > 0
        exp = alone[j].query(steps).cpu().numpy()
        np.testing.assert_array_equal(got, exp)
    st = sv.stats()
    assert st["queries"] == 200 and st["batches"] < 200
    # one query alone on the server gives the same result as in the mix
    j, steps = queries[0]
    got, _ = sv.poll(sv.submit(ids[j], steps))
    np.testing.assert_array_equal(got, alone[j].query(steps).cpu().numpy())
    for ds in alone:
        ds.close()
    sv.close()


def test_queue_full_timeouts_cancel_and_remove():
    data, direction, cfg = _datasets()[0]
    sv = G.Server(2 << 30, max_batch=8, queue_capacity=4, start_paused=True)
    did = sv.add_dataset(data, direction, cfg)
    steps = steps_log(128, 16)
    tickets = [sv.submit(did, steps) for _ in range(4)]
    with pytest.raises(G.GresError) as e:
        sv.submit(did, steps)
    assert e.value.status == EAGAIN                       # queue full
    assert sv.poll(tickets[0], timeout_us=0) is None      # not started
    assert sv.poll(tickets[0], timeout_us=2000) is None   # the wait runs out
    with pytest.raises(G.GresError) as e:
        sv.remove_dataset(did)
    assert e.value.status == EAGAIN                       # queries still pending
    sv.cancel(tickets[1])
    with pytest.raises(G.GresError):
        sv.poll(tickets[1], timeout_us=0)                 # gone
    sv.resume()
    ref = G.Dataset(data, direction, cfg).query(steps).cpu().numpy()
    for t in (tickets[0], tickets[2], tickets[3]):
        got, _ = sv.poll(t, timeout_us=-1)
        np.testing.assert_array_equal(got, ref)
    sv.remove_dataset(did)
    with pytest.raises(G.GresError) as e:
        sv.submit(did, steps)
    assert e.value.status == EINVAL
    sv.close()


def test_hbm_budget():
    with pytest.raises(G.GresError) as e:
        G.Server(1 << 20, max_batch=64, max_k=4096)      # smaller than the batch buffers
    assert e.value.status == ENOMEM
    small = make_dataset("uni", 3000, 3, bits=20, seed=1)
    big = make_dataset("ant", 400000, 6, bits=20, seed=2)    # skyline tiles of several MB
    budget = 1 << 20
    sv = G.Server(budget, max_batch=16, max_k=512)
    sid = sv.add_dataset(small)
    with pytest.raises(G.GresError) as e:
        sv.add_dataset(big)
    assert e.value.status == ENOMEM
    got, _ = sv.poll(sv.submit(sid, steps_log(100, 16)))
    np.testing.assert_array_equal(got, G.Dataset(small).query(steps_log(100, 16)).cpu().numpy())
    assert sv.stats()["device_bytes"] <= budget
    sv.close()


def test_queries_in_pieces():
    """Queries split into pieces of a few hundred targets give the same results; a query
    on a small skyline submitted after one on a large skyline finishes first."""
    rng = np.random.default_rng(7)
    dsets = _datasets()
    alone = [G.Dataset(data, direction, cfg) for data, direction, cfg in dsets]
    for chunk in (300, -1):
        sv = G.Server(8 << 30, max_batch=16, max_inflight=3, chunk_targets=chunk)
        ids = [sv.add_dataset(data, direction, cfg) for data, direction, cfg in dsets]
        queries = [(int(rng.integers(0, len(ids))), steps_log(int(rng.integers(64, 257)), 16)) for _ in range(60)]
        tickets = [sv.submit(ids[j], steps) for j, steps in queries]
        for t, (j, steps) in zip(tickets, queries):
            got, _ = sv.poll(t)
            np.testing.assert_array_equal(got, alone[j].query(steps).cpu().numpy())
        sv.close()
    # ordering: the largest skyline in many pieces, then the smallest
    sizes = [ds.S for ds in alone]
    big, small = int(np.argmax(sizes)), int(np.argmin(sizes))
    assert sizes[big] > 20 * 100
    sv = G.Server(8 << 30, max_batch=16, max_inflight=2, chunk_targets=100, start_paused=True)
    ids = [sv.add_dataset(data, direction, cfg) for data, direction, cfg in dsets]
    steps = steps_log(256, 16)
    tb = sv.submit(ids[big], steps)
    ts = sv.submit(ids[small], steps)
    sv.resume()
    got_s, lat_s = sv.poll(ts)
    got_b, lat_b = sv.poll(tb)
    assert lat_s < lat_b
    np.testing.assert_array_equal(got_b, alone[big].query(steps).cpu().numpy())
    np.testing.assert_array_equal(got_s, alone[small].query(steps).cpu().numpy())
    # a cancelled query in pieces ends cleanly: the dataset can be removed afterwards
    tc = sv.submit(ids[big], steps)
    sv.cancel(tc)
    with pytest.raises(G.GresError):
        sv.poll(tc, timeout_us=0)
    got, _ = sv.poll(sv.submit(ids[big], steps))
    np.testing.assert_array_equal(got, alone[big].query(steps).cpu().numpy())
    for _ in range(1000):
        try:
            sv.remove_dataset(ids[big])
            break
        except G.GresError as e:
            assert e.status == EAGAIN
            time.sleep(0.002)
    else:
        raise AssertionError("dataset still busy after its queries ended")
    sv.close()
    for ds in alone:
        ds.close()

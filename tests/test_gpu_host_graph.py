"""GPU: the host-buffer entry point's graph replay (pinned inputs).

Repeated gres_compute_host calls with the same pinned buffer, widths, plan and
workspace replay one captured graph; the results must stay those of the
oracle, also after new data is written into the same buffer and after the
widths change (a new capture).
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2412_02274_gb300 import gres as G
from paper_2412_02274_gb300.inputs import make_dataset, steps_log

pytestmark = pytest.mark.gpu


def _expect(data, steps, direction="min"):
    sky = O.skyline_bnl(data, direction)
    return sky, O.gres(data, steps, direction, candidates=sky, targets=sky)


def test_replays_follow_the_buffer_contents_and_the_widths():
    n, d = 6000, 3
    a = make_dataset("ant", n, d, bits=20, seed=1)
    b = make_dataset("uni", n, d, bits=20, seed=2)
    pinned = torch.empty((n, d), dtype=torch.int32).pin_memory()
    hs = torch.empty(n, dtype=torch.int64).pin_memory()
    hr = torch.empty(n, dtype=torch.int32).pin_memory()
    steps = steps_log(128, 16)
    ws = G.alloc_workspace(n, d, 256, host=True)
    stream = torch.cuda.current_stream()
    for data in (a, a, a, b, b, a):        # first call captures, the rest replay
        pinned.copy_(torch.from_numpy(data.view(np.int32)))
        sky, res = G.gres_compute_host(pinned, steps, G.MIN, ws=ws, out=(hs, hr), stream=stream)
        esky, eres = _expect(data, steps)
        np.testing.assert_array_equal(sky, esky)
        np.testing.assert_array_equal(res, eres)
    for steps2 in (steps_log(256, 16), steps_log(64, 12)):   # other widths: a new capture
        for _ in range(2):
            sky, res = G.gres_compute_host(pinned, steps2, G.MIN, ws=ws, out=(hs, hr), stream=stream)
            esky, eres = _expect(a, steps2)
            np.testing.assert_array_equal(res, eres)
    # larger-is-better and another plan on the same buffer
    for _ in range(2):
        sky, res = G.gres_compute_host(pinned, steps, G.MAX, G.plan(G.PART_SLICED, p=8), ws=ws, out=(hs, hr),
                                       stream=stream)
        esky, eres = _expect(a, steps, "max")
        np.testing.assert_array_equal(sky, esky)
        np.testing.assert_array_equal(res, eres)


@pytest.mark.parametrize("pinned_out", [True, False])
def test_replays_with_more_or_fewer_results_than_the_capture(pinned_out):
    """The graph copies back as many results as the capturing call had (pinned result buffers):
    replays with a larger skyline copy the rest, smaller ones stop at S. Unpinned result buffers
    take the plain copies."""
    n, d = 5000, 4
    small = make_dataset("uni", n, d, bits=20, seed=3)    # few skyline rows
    large = make_dataset("ant", n, d, bits=20, seed=4)    # many
    pinned = torch.empty((n, d), dtype=torch.int32).pin_memory()
    if pinned_out:
        out = (torch.empty(n, dtype=torch.int64).pin_memory(), torch.empty(n, dtype=torch.int32).pin_memory())
    else:
        out = (torch.empty(n, dtype=torch.int64), torch.empty(n, dtype=torch.int32))
    steps = steps_log(96, 16)
    ws = G.alloc_workspace(n, d, 96, host=True)
    stream = torch.cuda.current_stream()
    sizes = []
    for data in (small, small, large, large, small, large):   # the first call captures with the small skyline
        pinned.copy_(torch.from_numpy(data.view(np.int32)))
        sky, res = G.gres_compute_host(pinned, steps, G.MIN, ws=ws, out=out, stream=stream)
        esky, eres = _expect(data, steps)
        np.testing.assert_array_equal(np.asarray(sky), esky)
        np.testing.assert_array_equal(np.asarray(res), eres)
        sizes.append(len(esky))
    assert sizes[2] > sizes[0]

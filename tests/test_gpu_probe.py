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

"""The seeded input generators against the recipe they state (no method arithmetic).

UNI is uniform on [0,1)^d; ANT moves uniform points onto the plane sum(x) = d/2
and offsets them along the plane's unit normal by N(0, sigma); CLU draws around
16 uniform centres with N(0, sigma_c^2 I). Values are min(floor(x 2^B), 2^B - 1).
"""
import numpy as np
import pytest

from paper_2412_02274_gb300.inputs import make_dataset

B = 20
ONE = float(1 << B)


def test_shape_type_range_and_determinism():
    for dist in ("uni", "ant", "clu"):
        a = make_dataset(dist, 5000, 5, bits=B, seed=3)
        b = make_dataset(dist, 5000, 5, bits=B, seed=3)
        c = make_dataset(dist, 5000, 5, bits=B, seed=4)
        assert a.shape == (5000, 5) and a.dtype == np.uint32 and a.flags["C_CONTIGUOUS"]
        assert int(a.max()) <= (1 << B) - 1
        assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert make_dataset("uni", 0, 3).shape == (0, 3)
    with pytest.raises(ValueError):
        make_dataset("nope", 10, 2)
    with pytest.raises(ValueError):
        make_dataset("uni", 10, 2, bits=33)


def test_uniform_moments():
    x = make_dataset("uni", 200000, 4, bits=B, seed=0) / ONE
    assert np.allclose(x.mean(axis=0), 0.5, atol=0.005)
    assert np.allclose(x.var(axis=0), 1.0 / 12.0, atol=0.002)
    # attributes independent
    c = np.corrcoef(x.T)
    assert np.abs(c - np.eye(4)).max() < 0.01


@pytest.mark.parametrize("d", [2, 4, 6])
def test_anticorrelated_offset_from_the_plane(d):
    sigma = 0.05
    x = make_dataset("ant", 200000, d, bits=B, seed=1, sigma=sigma) / ONE
    # signed distance from the plane sum(x) = d/2 along the unit normal
    off = (x.sum(axis=1) - d / 2.0) / np.sqrt(d)
    # clipping to [0, 1) moves a few points; the bulk follows N(0, sigma)
    assert abs(np.median(off)) < 0.1 * sigma
    q25, q75 = np.percentile(off, [25, 75])
    assert abs((q75 - q25) / 1.349 - sigma) < 0.1 * sigma
    # anticorrelated: on the plane every pair of attributes has correlation -1 / (d - 1)
    c = np.corrcoef(x.T)
    assert (c[~np.eye(d, dtype=bool)] < -0.75 / (d - 1)).all()


def test_clustered_around_sixteen_centres():
    x = make_dataset("clu", 100000, 3, bits=B, seed=2) / ONE
    # most points sit within a few cluster sigmas of one of at most 16 dense cells
    cells = np.floor(x / 0.1).astype(np.int64)
    keys = cells[:, 0] * 10000 + cells[:, 1] * 100 + cells[:, 2]
    _, counts = np.unique(keys, return_counts=True)
    top = np.sort(counts)[::-1]
    # 16 centres, each spread over at most 8 cells of side 0.1 (sigma_c = 0.02), hold nearly all
    assert top[:128].sum() > 0.95 * len(x)
    # the densest cell is far above the uniform density of 100 points per cell
    assert top[0] > 20 * len(x) / 1000

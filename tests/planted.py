"""Datasets whose skyline is known by construction (test helper).

``planted_skyline`` draws ``n_plane`` rows on the hyperplane
``sum(x) = (d - 1) * 2**span_bits`` and ``n_dom`` rows that each copy a
plane row and add a non-negative offset that is positive in at least one
attribute. Under smaller-is-better dominance (Def. 1):

* every offset row is dominated by the plane row it copies;
* nothing dominates a plane row, since a dominator has a strictly smaller
  attribute sum and no row has a sum below the plane's; plane rows that are
  equal do not dominate each other.

So the skyline is exactly the plane rows, at any size. The tests use this to
check large skylines (hundreds of thousands of rows, far more than the
oracle's pairwise skyline can do in seconds) against an exact expectation,
and check the construction itself against the oracle on small instances.
"""
from __future__ import annotations

import numpy as np


def planted_skyline(n_plane: int, n_dom: int, d: int, seed: int = 0, span_bits: int = 17,
                    offset_bits: int = 10):
    """``(data, sky)``: an ``(n_plane + n_dom, d)`` uint32 array in random row order
    and the ascending row numbers of its plane rows (its skyline)."""
    if d < 2:
        raise ValueError("d must be >= 2")
    rng = np.random.Generator(np.random.PCG64(seed))
    c = (d - 1) << span_bits
    head = rng.integers(0, 1 << span_bits, size=(n_plane, d - 1), dtype=np.int64)
    plane = np.concatenate([head, (c - head.sum(axis=1))[:, None]], axis=1)
    src = rng.integers(0, n_plane, size=n_dom)
    off = rng.integers(0, 1 << offset_bits, size=(n_dom, d), dtype=np.int64)
    off[np.arange(n_dom), rng.integers(0, d, size=n_dom)] += 1
    rows = np.concatenate([plane, plane[src] + off], axis=0)
    assert rows.min() >= 0 and rows.max() < (1 << 32)
    perm = rng.permutation(n_plane + n_dom)
    data = np.ascontiguousarray(rows[perm].astype(np.uint32))
    sky = np.flatnonzero(perm < n_plane).astype(np.int64)
    return data, sky

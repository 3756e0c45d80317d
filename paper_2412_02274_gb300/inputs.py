"""Seeded synthetic inputs: datasets and step sequences.

This module is shared by the CUDA path, the oracle tests and the benchmark. It
holds no arithmetic of the method itself (no dominance, no projection, no
skyline): it only draws numbers and turns them into fixed-point ``uint32``
tuples and integer step lists.

Value encoding: a real value ``x`` in ``[0, 1)`` (the paper's domain for the
synthetic data, Sec. 4) becomes ``v = min(floor(x * 2**B), 2**B - 1)``.

Distributions (Sec. 4 uses UNI and ANT; CLU is an added mix member):

* ``uni``  -- ``x ~ U[0,1)^d``.
* ``ant``  -- anticorrelated: ``u ~ U[0,1)^d`` moved onto the plane
  ``sum(x) = d/2`` along the all-ones direction, then offset along the unit
  normal by ``o ~ N(0, sigma)``; clipped to ``[0, 1)``.
* ``clu``  -- 16 centres ``~ U[0,1)^d``; each point picks a centre uniformly and
  adds ``N(0, sigma_c^2 I)``; clipped to ``[0, 1)``.

Step sequences are ascending integer cell widths ``delta_0 < ... < delta_{K-1}``.
``steps_log(K, E)`` spreads K widths over ``1 .. 2**E`` on a log scale with
every width of the form ``j * 2**k`` (``j < 64``); ``steps_linear(K, w)`` is
``w, 2w, ..., K*w``.
"""
from __future__ import annotations

import numpy as np

__all__ = ["make_dataset", "steps_log", "steps_linear", "DISTRIBUTIONS"]

DISTRIBUTIONS = ("uni", "ant", "clu")

_ONE_BELOW = np.nextafter(1.0, 0.0)


def _to_fixed(x: np.ndarray, bits: int) -> np.ndarray:
    x = np.clip(x, 0.0, _ONE_BELOW)
    v = np.floor(x * float(1 << bits))
    v = np.minimum(v, float((1 << bits) - 1))
    return np.ascontiguousarray(v.astype(np.uint32))


def make_dataset(dist: str, n: int, d: int, bits: int = 20, seed: int = 0,
                 sigma: float = 0.05, clusters: int = 16,
                 cluster_sigma: float = 0.02) -> np.ndarray:
    """Return an ``(n, d)`` C-contiguous ``uint32`` array of fixed-point tuples."""
    if dist not in DISTRIBUTIONS:
        raise ValueError(f"unknown distribution {dist!r}")
    if not (1 <= bits <= 32):
        raise ValueError("bits must be in [1, 32]")
    rng = np.random.Generator(np.random.PCG64(seed))
    if n == 0:
        return np.zeros((0, d), dtype=np.uint32)
    if dist == "uni":
        x = rng.random((n, d))
    elif dist == "ant":
        u = rng.random((n, d))
        x = u + ((d / 2.0 - u.sum(axis=1, keepdims=True)) / d)
        o = rng.normal(0.0, sigma, size=(n, 1))
        x = x + o / np.sqrt(d)
    else:
        centres = rng.random((clusters, d))
        pick = rng.integers(0, clusters, size=n)
        x = centres[pick] + rng.normal(0.0, cluster_sigma, size=(n, d))
    return _to_fixed(x, bits)


def _iroot_floor(value: int, r: int) -> int:
    """Largest integer c with c**r <= value (value >= 0, r >= 1)."""
    if value < 2 or r == 1:
        return value
    lo, hi = 1, 1 << (value.bit_length() // r + 1)
    while lo < hi:
        mid = (lo + hi + 1) // 2
        if mid ** r <= value:
            lo = mid
        else:
            hi = mid - 1
    return lo


def _keep_top_bits(c: int, keep: int = 6) -> int:
    b = c.bit_length()
    if b <= keep:
        return c
    return (c >> (b - keep)) << (b - keep)


def steps_log(k: int, e: int = 16) -> np.ndarray:
    """K strictly ascending widths from 1 to ``2**e``, each ``j * 2**s`` with ``j < 64``.

    ``c_i = top6(floor(2**(e*i/(K-1))))`` (an exact integer root), then
    ``delta_0 = 1`` and ``delta_i = max(delta_{i-1} + 1, c_i)``.
    """
    if k < 1:
        raise ValueError("k must be >= 1")
    out = [1]
    for i in range(1, k):
        c = _keep_top_bits(_iroot_floor(1 << (e * i), k - 1))
        out.append(max(out[-1] + 1, c))
    arr = np.asarray(out, dtype=np.uint64)
    if arr.max() > 0xFFFFFFFF:
        raise ValueError("step exceeds uint32")
    return arr.astype(np.uint32)


def steps_linear(k: int, width: int) -> np.ndarray:
    """``width, 2*width, ..., k*width``."""
    if k < 1 or width < 1 or k * width > 0xFFFFFFFF:
        raise ValueError("bad linear step list")
    return (np.arange(1, k + 1, dtype=np.uint64) * width).astype(np.uint32)

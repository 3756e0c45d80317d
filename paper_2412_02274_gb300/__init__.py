"""Grid resistance (gres) of skyline tuples on GB300 (sm_103a).

The compute path is the C-ABI library ``libgres`` (hand-written CUDA kernels);
``paper_2412_02274_gb300.gres`` is its thin ctypes binding. Importing this
package loads nothing: the library is loaded on first use and a missing or
unloadable library raises an error (there is no CPU fallback).
"""
__all__ = ["inputs"]

"""A CPU restatement of the grid-dominance kernel's search, for its counters (test helper).

The library's GRES_FLAG_COUNT_TESTS counters feed the benchmark's roofline numerator:
d_tests[0] counts lane-tests (32 per warp-wide test of one candidate row at the 32
widths of a slot) and d_tests[1] pruning checks (32 per warp-wide look at 32
super-tile minima, 32 tile minima or 32 candidate rows). `count_search` walks the
same search in the same order -- super-tiles and tiles best-first by their excess
bound with ties to the lower lane, the rows of a tile in index order, slots from
the first that can matter up to the current best -- and counts the same events, so
that a test can pin the kernel's counters exactly on small inputs.

It also returns each target's first exit step, which must equal the oracle's (the
search is exact), so the model is checked against Def. 2 as well.

Inputs: the candidate rows in the kernel's tile order (canonical values: v for
smaller-is-better, ~v for larger-is-better), the widths, the direction, the slot
count. Tiles hold 32 rows, super-tiles 32 tiles; rows past the end are sentinel
rows (all ones), which never dominate.
"""
from __future__ import annotations

import numpy as np

FULL = 0xFFFFFFFF
NOKEY = 0xFFFFFFFF


def layout(cand_rows: np.ndarray):
    """(padded rows, tile minima, super-tile minima) of canonical rows in tile order."""
    S, d = cand_rows.shape
    T = (S + 31) // 32
    pad = np.full((T * 32, d), FULL, dtype=np.uint64)
    pad[:S] = cand_rows
    tmin = pad.reshape(T, 32, d).min(axis=1)
    T2 = (T + 31) // 32
    tp = np.full((T2 * 32, d), FULL, dtype=np.uint64)
    tp[:T] = tmin
    smin = tp.reshape(T2, 32, d).min(axis=1)
    return pad, tmin, smin


def _bound(mins: np.ndarray, t: np.ndarray):
    """Per row of mins: (max_i (m_i - t_i)^+, any_i m_i < t_i)."""
    ex = np.where(mins > t, mins - t, 0).max(axis=1)
    can = (mins < t).any(axis=1)
    return ex, can


def _cell(t: np.ndarray, delta: int, direction: int):
    """Canonical cell [lo, hi] of canonical target t at width delta (per attribute)."""
    raw = (~t & FULL) if direction else t
    lv = (raw // delta) * delta
    uv = np.minimum(lv + (delta - 1), FULL)
    if direction:
        return (~uv & FULL), (~lv & FULL)
    return lv, uv


def count_search(cand_rows, widths, direction: int = 0, slots: int = 8, pid=None, nparts: int = 0):
    """(first exit step per candidate position, lane-tests, pruning checks), plus, with pid
    (the partition number of every candidate position) and nparts, the per-partition split
    of GRES_FLAG_COUNT_PARTS: an (nparts, 4) array of (local lane-tests, local row checks,
    cross lane-tests, cross row checks) by the target's partition."""
    cand_rows = np.asarray(cand_rows, dtype=np.uint64)
    widths = [int(w) for w in widths]
    S, d = cand_rows.shape
    K = len(widths)
    WS = 32 * slots
    pad, tmin, smin = layout(cand_rows)
    T = len(tmin)
    T2 = len(smin)
    tests = checks = 0
    out = np.empty(S, dtype=np.int64)
    split = np.zeros((max(nparts, 1), 4), dtype=np.int64)
    pad_pid = np.full(T * 32, -1, dtype=np.int64)
    if pid is not None:
        pad_pid[:S] = np.asarray(pid, dtype=np.int64)
    for i in range(S):
        t = cand_rows[i]
        result = K
        for w0 in range(0, K, WS):
            wcount = min(WS, K - w0)
            wsteps = [widths[w0 + j] if w0 + j < K else FULL for j in range(WS)]
            best = wcount
            wmax = wsteps[wcount - 1]
            qshift = (wmax.bit_length() - 24) if wmax >> 24 else 0
            wl = wsteps[best - 1] if best > 0 else 0
            wlq = min(wl >> qshift, 0x7FFFFFF)
            slot_top = [wsteps[32 * l + 31] if (l < slots - 1 and 32 * l + 31 < wcount) else FULL
                        for l in range(32)]

            def key(ex, lane):
                return (min(int(ex) >> qshift, 0x7FFFFFF) << 5) | lane

            s0 = 0
            while s0 < T2 and best > 0:
                ids = [s0 + l for l in range(32)]
                skey, sex = [NOKEY] * 32, [FULL] * 32
                for l, s in enumerate(ids):
                    if s < T2:
                        ex, can = _bound(smin[s:s + 1], t)
                        if can[0] and ex[0] < wl:
                            sex[l], skey[l] = int(ex[0]), key(ex[0], l)
                checks += 32
                while True:
                    mk = min(skey)
                    if mk == NOKEY or (mk >> 5) > wlq:
                        break
                    sl = mk & 31
                    skey[sl] = NOKEY
                    if sex[sl] >= wl:
                        continue
                    sup = s0 + sl
                    tkey, tex = [NOKEY] * 32, [FULL] * 32
                    for l in range(32):
                        tile = sup * 32 + l
                        if tile < T:
                            ex, can = _bound(tmin[tile:tile + 1], t)
                            if can[0] and ex[0] < wl:
                                tex[l], tkey[l] = int(ex[0]), key(ex[0], l)
                    checks += 32
                    while True:
                        tk = min(tkey)
                        if tk == NOKEY or (tk >> 5) > wlq:
                            break
                        tl = tk & 31
                        tkey[tl] = NOKEY
                        if tex[tl] >= wl:
                            continue
                        r0 = (sup * 32 + tl) * 32
                        rows = pad[r0:r0 + 32]
                        e_r, can_r = _bound(rows, t)
                        checks += 32
                        if pid is not None:
                            loc = int((pad_pid[r0:r0 + 32] == pad_pid[i]).sum())
                            split[pad_pid[i], 1] += loc
                            split[pad_pid[i], 3] += 32 - loc
                        elig = [c for c in range(32) if can_r[c] and e_r[c] < wl]
                        for c in elig:
                            ec = int(e_r[c])
                            if ec >= wl:
                                continue
                            cv = rows[c]
                            jlo = sum(1 for l in range(32) if slot_top[l] <= ec)
                            jhi = (best - 1) >> 5
                            for j in range(jlo, jhi + 1):
                                tests += 32
                                if pid is not None:
                                    split[pad_pid[i], 0 if pad_pid[r0 + c] == pad_pid[i] else 2] += 32
                                hit = None
                                for lane in range(32):
                                    k = w0 + 32 * j + lane
                                    if k >= K:
                                        continue
                                    lo, hi = _cell(t, widths[k], direction)
                                    if np.all(cv <= hi) and np.any(cv < lo):
                                        hit = lane
                                        break
                                if hit is not None:
                                    best = min(best, 32 * j + hit)
                                    if best > 0:
                                        wl = wsteps[best - 1]
                                        wlq = min(wl >> qshift, 0x7FFFFFF)
                                    break
                            if best == 0:
                                break
                        if best == 0:
                            break
                    if best == 0:
                        break
                s0 += 32
            if best < wcount:
                result = w0 + best
                break
        out[i] = result
    if pid is not None:
        return out, tests, checks, split
    return out, tests, checks

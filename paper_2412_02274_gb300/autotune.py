"""Plan autotuner for gres problems.

A plan (``gres_plan_cfg``: how the skyline candidates are grouped into tiles --
Grid / Angular / Sliced partitioning of Sec. 3.1 or none -- and the kernel's
per-warp width slots) changes the speed of a gres computation, never its
result. The tuner times a fixed list of candidate plans on sample problems of
each size class (attribute count d and the power-of-two bucket of the row
count n) with CUDA events, keeps the plan with the lowest score per class
(the whole call, or its cost inside a gres_batch, see score()), and
afterwards hands out plans by class. Classes it has not seen take the nearest tuned class
with the same d, else the library default.

The timing function is a parameter, so that the selection logic runs (and is
tested) without a GPU.
"""
from __future__ import annotations

import json
from dataclasses import dataclass

import numpy as np

from . import gres as G


@dataclass(frozen=True)
class Candidate:
    name: str
    scheme: int
    m: int = 0
    p: int = 0
    slots: int = 8
    gres_reps: bool = False

    def cfg(self) -> G.PlanCfg:
        return G.plan(self.scheme, m=self.m, p=self.p, slots=self.slots, gres_reps=self.gres_reps)


def default_candidates() -> list[Candidate]:
    out = []
    for slots in (8, 4):
        out += [Candidate(f"grid-auto-s{slots}", G.PART_GRID, slots=slots),
                Candidate(f"grid-m2-s{slots}", G.PART_GRID, m=2, slots=slots),
                Candidate(f"grid-m3-s{slots}", G.PART_GRID, m=3, slots=slots),
                Candidate(f"angular-auto-s{slots}", G.PART_ANGULAR, slots=slots),
                Candidate(f"sliced-p64-s{slots}", G.PART_SLICED, p=64, slots=slots),
                Candidate(f"none-s{slots}", G.PART_NONE, slots=slots)]
    # Representative Filtering in the gres stage on the usual winners
    out += [Candidate(f"{c.name}-reps", c.scheme, c.m, c.p, c.slots, True)
            for c in out if c.name.startswith(("grid-auto", "grid-m2", "grid-m3", "none"))]
    return out


def size_class(n: int, d: int) -> tuple[int, int]:
    """(d, b) with 2^(b-1) <= n < 2^b (b = 0 for n = 0)."""
    return int(d), int(n).bit_length()


def cuda_event_timer(repeats: int = 3):
    """Median CUDA-event times (ms) of gres_compute(data, steps, direction, cfg) after one
    warm-up: {"total", "skyline", "partition", "dominance"}."""
    def run(data, steps, direction, cfg, ws):
        import torch
        stream = torch.cuda.current_stream()
        G.gres_compute(data, steps, direction, cfg, ws=ws, sync=False, stream=stream)
        rec = {"total": [], "skyline": [], "partition": [], "dominance": []}
        for _ in range(repeats):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            G.timing_enable(True)
            a.record(stream)
            G.gres_compute(data, steps, direction, cfg, ws=ws, sync=False, stream=stream)
            b.record(stream)
            b.synchronize()
            stages = G.timing_read()
            G.timing_enable(False)
            rec["total"].append(a.elapsed_time(b))
            for k in ("skyline", "partition", "dominance"):
                rec[k].append(stages[k][0])
        return {k: float(np.median(v)) for k, v in rec.items()}
    return run


def score(times, objective: str = "alone", concurrency: int = 16) -> float:
    """The number the tuner minimises. ``alone``: the whole call. ``batch``: the call as
    part of gres_batch, where the skyline and partitioning stages of many instances run
    on ``concurrency`` forked streams at once and the grid-dominance kernels of all
    instances share one launch: dominance + (skyline + partition) / concurrency."""
    if not isinstance(times, dict):
        return float(times)
    if objective == "batch":
        return times["dominance"] + (times["skyline"] + times["partition"]) / concurrency
    return times["total"]


class Autotuner:
    """Fastest candidate plan per size class, chosen by timing sample problems."""

    def __init__(self, candidates: list[Candidate] | None = None, timer=None, objective: str = "alone",
                 concurrency: int = 16, default: str = "grid-auto-s8", margin: float = 0.05):
        if objective not in ("alone", "batch"):
            raise ValueError("objective must be 'alone' or 'batch'")
        self.candidates = list(candidates or default_candidates())
        self._by_name = {c.name: c for c in self.candidates}
        self.timer = timer
        self.objective = objective
        self.concurrency = concurrency
        # a candidate replaces the library's default plan only if it scores at least
        # `margin` lower: single timings of the sample problems move by a few percent
        self.default = default if default in self._by_name else None
        self.margin = margin
        self.table: dict[tuple[int, int], str] = {}
        self.timings: dict[tuple[int, int], dict[str, float]] = {}

    def tune(self, problems, steps, direction: int = G.MIN, samples_per_class: int = 2,
             workspace=None) -> dict:
        """Times every candidate on up to ``samples_per_class`` problems of each class.

        ``problems``: (n, d) arrays as the timer takes them (CUDA tensors for the
        default timer). ``workspace(n, d, k)`` makes a workspace for a sample (the
        default allocates one per sample). Returns the class -> plan name table."""
        timer = self.timer or cuda_event_timer()
        k = len(steps)
        groups: dict[tuple[int, int], list] = {}
        for x in problems:
            n, d = int(x.shape[0]), int(x.shape[1])
            groups.setdefault(size_class(n, d), []).append(x)
        for cls, members in sorted(groups.items()):
            # the largest members of the class (the ones whose time counts most)
            members = sorted(members, key=lambda x: -int(x.shape[0]))[:samples_per_class]
            total = {c.name: 0.0 for c in self.candidates}
            for x in members:
                n, d = int(x.shape[0]), int(x.shape[1])
                ws = workspace(n, d, k) if workspace else (G.alloc_workspace(n, d, k) if self.timer is None else None)
                for c in self.candidates:
                    total[c.name] += score(timer(x, steps, direction, c.cfg(), ws), self.objective,
                                           self.concurrency)
            self.timings[cls] = total
            best = min(self.candidates, key=lambda c: (total[c.name], c.name)).name
            if self.default and total[best] > (1.0 - self.margin) * total[self.default]:
                best = self.default
            self.table[cls] = best
        return dict(self.table)

    def plan_for(self, n: int, d: int) -> G.PlanCfg:
        """The tuned plan of (n, d)'s class; the nearest tuned class of the same d; else the default."""
        cls = size_class(n, d)
        name = self.table.get(cls)
        if name is None:
            same_d = [c for c in self.table if c[0] == cls[0]]
            if not same_d:
                return G.plan()
            near = min(same_d, key=lambda c: (abs(c[1] - cls[1]), c[1]))
            name = self.table[near]
        return self._by_name[name].cfg()

    def to_json(self) -> str:
        return json.dumps({"candidates": [c.__dict__ for c in self.candidates],
                           "table": [[d, b, name] for (d, b), name in sorted(self.table.items())],
                           "timings_ms": [[d, b, t] for (d, b), t in sorted(self.timings.items())]})

    @classmethod
    def from_json(cls, text: str) -> "Autotuner":
        obj = json.loads(text)
        tuner = cls([Candidate(**c) for c in obj["candidates"]])
        tuner.table = {(int(d), int(b)): name for d, b, name in obj["table"]}
        tuner.timings = {(int(d), int(b)): t for d, b, t in obj.get("timings_ms", [])}
        return tuner

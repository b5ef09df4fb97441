"""Autotuned schedule tables.

A schedule is the radix and tile plan of one axis's pass kernel (listed in
include/spstd.h): the library times the candidates on a live context
(spstd_tune) or over a batch's members (spstd_batch_tune) and keeps the
fastest.  This module keeps those choices in a JSON table keyed by the grid
shape and precision, so a later process can apply them without timing again:

    {"version": 1,
     "entries": {"3d:256x256x256:fp32": {"schedule": [0, 0, 0],
                                         "ms": [[...], [...], [...]]}}}

Only argument marshalling lives here; the timing runs in the library.
"""
from __future__ import annotations

import json
import os
from typing import Dict, List, Optional, Sequence

VERSION = 1


def shape_key(dims: int, n: Sequence[int], precision: int) -> str:
    """Table key of a grid: '<dims>d:<n0>x<n1>...:fp<precision>'."""
    return f"{int(dims)}d:{'x'.join(str(int(v)) for v in list(n)[: int(dims)])}:fp{int(precision)}"


def solver_key(solver) -> str:
    cfg = solver.cfg
    return shape_key(cfg.dims, [cfg.n[a] for a in range(cfg.dims)], cfg.precision)


class ScheduleTable:
    def __init__(self, entries: Optional[Dict[str, dict]] = None):
        self.entries: Dict[str, dict] = dict(entries or {})

    @classmethod
    def load(cls, path: str) -> "ScheduleTable":
        if not os.path.exists(path):
            return cls()
        with open(path) as f:
            doc = json.load(f)
        if doc.get("version") != VERSION:
            raise ValueError(f"{path}: schedule table version {doc.get('version')} (expected {VERSION})")
        return cls(doc.get("entries", {}))

    def save(self, path: str) -> None:
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            json.dump({"version": VERSION, "entries": self.entries}, f, indent=1, sort_keys=True)
        os.replace(tmp, path)

    def lookup(self, key: str) -> Optional[List[int]]:
        e = self.entries.get(key)
        return list(e["schedule"]) if e else None

    def record(self, key: str, schedule: Sequence[int], ms=None) -> None:
        e = {"schedule": [int(v) for v in schedule]}
        if ms is not None:
            e["ms"] = [[round(float(t), 6) for t in row] for row in ms]
        self.entries[key] = e

    def apply(self, solver) -> bool:
        """Sets the solver's schedules from the table; False if the shape is
        absent or an entry is not a candidate on this build."""
        sched = self.lookup(solver_key(solver))
        if sched is None:
            return False
        dims = solver.cfg.dims
        for ax in range(dims):
            if sched[ax] not in solver.spstd_schedule_candidates(ax):
                return False
        for ax in range(dims):
            solver.spstd_set_schedule(ax, sched[ax])
        return True

    def tune(self, solver, reps: int = 20) -> List[int]:
        """Times the solver's candidates (spstd_tune), records and returns the choice."""
        ms = solver.spstd_tune(reps)
        dims = solver.cfg.dims
        sched = [solver.spstd_get_schedule(ax) for ax in range(dims)]
        self.record(solver_key(solver), sched, ms[:dims])
        return sched

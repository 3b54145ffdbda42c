"""Autotuner of the kernel layouts.

The paper's library is built in size-specialized variants chosen for the
target (Sec. 5.1: HP2, HP2F).  Here every batched routine has several kernel
layouts -- problems per CTA, lanes per problem, a split k-loop, a blocked
factorization -- and a built-in rule picks one from the order and the batch
size.  ``tune`` times every layout that has a kernel for a given (routine,
order, batch) on the caller's own operands, keeps the fastest in the
library's layout table (bf_layout_set) and returns the timings; ``Table``
records the choices and applies or saves them as JSON, so that a later
process reuses them without timing again.

Timing is on the device, with CUDA events on the launching stream, after
warm-up launches; the choice is the layout with the smallest median.
"""
from __future__ import annotations

import json
from dataclasses import dataclass, field

from ._abi import load

ROUTINE_IDS = {"dgemm_nt": 0, "dsyrk_ln": 1, "dpotrf_l": 2, "dtrsm_rltn": 3, "dsyrk_dpotrf_ln": 4, "dgetrf": 5,
              "dgelqf": 6}

LAYOUT_NAMES = {
    "dgemm_nt": {1: "ks1", 2: "ks2", 3: "ks4"},
    "dsyrk_ln": {1: "ks1", 2: "ks2", 3: "ks4"},
    "dpotrf_l": {1: "tiny", 2: "small_g2", 3: "small_g4", 4: "small_g8", 5: "small_g16", 6: "small_g32", 7: "rows",
                 8: "latency", 9: "split", 10: "blocked", 11: "rows8"},
    "dtrsm_rltn": {1: "rows", 2: "latency_r2", 3: "latency_r4", 4: "latency_r8"},
    "dgetrf": {1: "warp", 2: "rows", 3: "blocked", 4: "blocked16"},
    "dgelqf": {1: "warp", 2: "rows", 3: "blocked", 4: "blocked16"},
}
LAYOUT_NAMES["dsyrk_dpotrf_ln"] = LAYOUT_NAMES["dpotrf_l"]
GELQF_ONE_CTA_MAX_MN = 16384  # the one-CTA gelqf kernels hold m * n <= 16384 doubles


def _rid(routine: str) -> int:
    if routine not in ROUTINE_IDS:
        raise ValueError(f"unknown routine {routine!r}")
    return ROUTINE_IDS[routine]


def _order(routine: str, m: int, n: int) -> int:
    return n if routine in ("dtrsm_rltn", "dgelqf") else m


def rule_layout(routine: str, batch: int, m: int, n: int = 0, k: int = 0) -> int:
    """The layout the built-in rule picks (the table entry is cleared first)."""
    lib = load()
    order = _order(routine, m, n)
    lib.bf_layout_set(_rid(routine), order, batch, 0)
    return lib.bf_layout_get(_rid(routine), batch, m, n, k)


def current_layout(routine: str, batch: int, m: int, n: int = 0, k: int = 0) -> int:
    """The layout a call with these sizes uses now (forced, else the rule's)."""
    return load().bf_layout_get(_rid(routine), batch, m, n, k)


def candidates(routine: str, order: int, batch: int, m: int | None = None) -> list[int]:
    """Layouts that have a kernel for this order (leaves the entry at the rule).
    gelqf is keyed by its column count; with the row count `m` given, the
    one-CTA layouts that cannot hold an m x order matrix are left out."""
    lib = load()
    rid = _rid(routine)
    out = [lay for lay in range(1, lib.bf_layout_count(rid)) if lib.bf_layout_set(rid, order, batch, lay) == 0]
    lib.bf_layout_set(rid, order, batch, 0)
    if routine == "dgelqf" and m is not None and m * order > GELQF_ONE_CTA_MAX_MN:
        out = [lay for lay in out if LAYOUT_NAMES[routine][lay].startswith("blocked")]
    return out


@dataclass
class Choice:
    routine: str
    order: int
    batch: int
    layout: int
    rule: int
    ms: dict = field(default_factory=dict)

    def as_dict(self):
        names = LAYOUT_NAMES[self.routine]
        return {"layout": names.get(self.layout, self.layout), "rule_layout": names.get(self.rule, self.rule),
                "layout_ms": {names.get(k, k): round(v, 4) for k, v in sorted(self.ms.items())}}


def _median(xs):
    xs = sorted(xs)
    return xs[len(xs) // 2]


def tune(routine: str, batch: int, m: int, n: int, k: int, run, stream=None, reps: int = 5, warmup: int = 2,
         skip=None) -> Choice:
    """Time every layout of `routine` for these sizes with `run()` (one call
    of the routine on `stream`), keep the fastest in the layout table and
    return the timings (ms per call, median of `reps`).  `skip(layout)` may
    leave a candidate out (e.g. one known to be orders of magnitude slower
    for the batch)."""
    import torch

    lib = load()
    rid = _rid(routine)
    order = _order(routine, m, n)
    stream = stream if stream is not None else torch.cuda.current_stream()
    rule = rule_layout(routine, batch, m, n, k)
    times = {}
    for lay in candidates(routine, order, batch, m):
        if skip is not None and lay != rule and skip(lay):
            continue
        lib.bf_layout_set(rid, order, batch, lay)
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                run()
            ts = []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                run()
                e1.record(stream)
                ts.append((e0, e1))
            stream.synchronize()
        times[lay] = _median([a.elapsed_time(b) for a, b in ts])
    best = min(times, key=times.get)
    lib.bf_layout_set(rid, order, batch, best)
    return Choice(routine, order, batch, best, rule, times)


class Table:
    """Tuned choices: (routine, order, batch) -> layout."""

    def __init__(self):
        self.entries: dict[tuple[str, int, int], int] = {}

    def add(self, c: Choice):
        self.entries[(c.routine, c.order, c.batch)] = c.layout

    def apply(self):
        lib = load()
        for (routine, order, batch), lay in self.entries.items():
            r = lib.bf_layout_set(_rid(routine), order, batch, lay)
            if r != 0:
                raise RuntimeError(f"bf_layout_set({routine}, {order}, {batch}, {lay}) returned {r}")

    def save(self, path: str):
        with open(path, "w") as f:
            json.dump([{"routine": r, "order": o, "batch": b, "layout": lay}
                       for (r, o, b), lay in sorted(self.entries.items())], f, indent=1)

    @classmethod
    def load(cls, path: str) -> "Table":
        t = cls()
        with open(path) as f:
            for e in json.load(f):
                t.entries[(e["routine"], int(e["order"]), int(e["batch"]))] = int(e["layout"])
        return t

"""Lane-count autotuning of batched solves (lrp_group).

A batch solved as `lanes` concurrent sub-batches returns exactly the results of
one plan (same per-problem kernels and arithmetic), so the lane count is a pure
performance knob: more lanes let one lane's latency-bound per-problem kernels
overlap another lane's tall products, at the cost of smaller launches.  The
autotuner times each candidate lane count on the caller's own inputs (one
untimed warm-up that also captures the iteration graphs, then timed runs with
CUDA events on the caller's stream) and keeps the fastest in a JSON table keyed
by precision, n, right-hand-side rank class and batch size.  Only the timing
runs touch the GPU; the selection and the table are host logic.
"""
from __future__ import annotations

import json
import os
import statistics
from typing import Callable, Dict, Iterable, List, Optional, Tuple

DEFAULT_LANES = (1, 2, 4, 8)
TIE = 0.01  # candidates within 1% of the fastest count as ties


def rank_class(r_f: int) -> int:
    """Right-hand-side rank bucket: the smallest power of two >= r_f (>= 1)."""
    c = 1
    while c < max(1, int(r_f)):
        c <<= 1
    return c


def table_key(precision: str, n: int, r_f: int, batch: int) -> str:
    return f"{precision}/n{int(n)}/rf{rank_class(r_f)}/b{int(batch)}"


def candidate_lanes(batch: int, candidates: Iterable[int] = DEFAULT_LANES) -> List[int]:
    """Lane counts worth timing: every lane gets at least one problem."""
    return sorted({int(c) for c in candidates if 1 <= int(c) <= int(batch)})


def choose(times: Dict[int, List[float]]) -> int:
    """The lane count with the smallest median time; candidates within TIE of
    it count as ties, which go to the fewest lanes (less memory, fewer
    streams)."""
    med = {lanes: statistics.median(ts) for lanes, ts in times.items() if ts}
    if not med:
        raise ValueError("no timed candidate")
    best = min(med.values())
    return min(lanes for lanes, m in med.items() if m <= best * (1.0 + TIE))


def tune_lanes(measure: Callable[[int], List[float]], batch: int,
               candidates: Iterable[int] = DEFAULT_LANES) -> Tuple[int, Dict[int, List[float]]]:
    """measure(lanes) -> timed runs (ms) of one batch at that lane count;
    returns the chosen lane count and every candidate's times."""
    times = {lanes: list(measure(lanes)) for lanes in candidate_lanes(batch, candidates)}
    return choose(times), times


class TuneTable:
    """Chosen lane counts, persisted as JSON ({key: {"lanes": L, "ms": {L: median}}})."""

    def __init__(self, path: Optional[str] = None):
        self.path = path
        self.entries: Dict[str, dict] = {}
        if path and os.path.exists(path):
            with open(path) as f:
                self.entries = json.load(f)

    def get(self, precision: str, n: int, r_f: int, batch: int) -> Optional[int]:
        e = self.entries.get(table_key(precision, n, r_f, batch))
        return int(e["lanes"]) if e else None

    def put(self, precision: str, n: int, r_f: int, batch: int, lanes: int,
            times: Dict[int, List[float]]) -> None:
        self.entries[table_key(precision, n, r_f, batch)] = {
            "lanes": int(lanes), "ms": {str(k): statistics.median(v) for k, v in times.items() if v}}

    def save(self) -> None:
        if not self.path:
            return
        tmp = self.path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(self.entries, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


def autotune_group(n: int, tol: float, max_rank: int, inputs, precision: str = "mixed",
                   candidates: Iterable[int] = DEFAULT_LANES, reps: int = 3,
                   table: Optional[TuneTable] = None, stream=None, **group_kw):
    """Lane count for solving `inputs` (a list of (U_f, s_f, V_f) device
    tensors, one problem each) with lrp_group.  A table hit returns at once;
    otherwise each candidate gets its own group (created, warmed up, timed
    `reps` times, closed before the next, so that only one workspace is held)
    and the choice is recorded in the table.  Returns (lanes, {lanes: [ms]})."""
    import torch

    from .api import Group
    batch = len(inputs)
    r_f = max(int(U.shape[1]) for U, _, _ in inputs)
    if table is not None:
        hit = table.get(precision, n, r_f, batch)
        if hit is not None:
            return hit, {}
    s = torch.cuda.current_stream() if stream is None else stream

    def measure(lanes: int) -> List[float]:
        g = Group(n, tol, max_rank, lanes=lanes, precision=precision, batch=batch, max_rhs_rank=r_f, **group_kw)
        try:
            outs = [g.alloc_outputs() for _ in inputs]
            g.solve_batch_into(inputs, outs, s)  # warm-up: workspace touched, graphs captured
            torch.cuda.synchronize()
            ms = []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(s)
                g.solve_batch_into(inputs, outs, s)
                e1.record(s)
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            return ms
        finally:
            g.close()

    lanes, times = tune_lanes(measure, batch, candidates)
    if table is not None:
        table.put(precision, n, r_f, batch, lanes, times)
        table.save()
    return lanes, times

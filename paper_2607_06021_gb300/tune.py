"""Autotuning of batched solves: lane count, loop placement and two launch
shapes (lrp_group, lrp_opts).

A batch solved as `lanes` concurrent sub-batches returns exactly the results of
one plan (same per-problem kernels and arithmetic), and a plan whose iteration
loops run on the device (`loop_on_device`, conditional graph nodes) returns
exactly the results of the host-driven loop.  Both are therefore pure
performance knobs: more lanes let one lane's latency-bound per-problem kernels
overlap another lane's tall products, at the cost of smaller launches; device
loops remove the host's read between iterations but launch every iteration over
the whole batch (finished problems exit at once instead of being compacted
away).  The autotuner times each candidate configuration on the caller's own
inputs (one untimed warm-up that also captures the graphs, then timed runs with
CUDA events on the caller's stream) and keeps the fastest in a JSON table keyed
by precision, n, right-hand-side rank class and batch size.  Only the timing
runs touch the GPU; the selection and the table are host logic.

The launch shapes are tuned next, one at a time at the chosen (lanes, loop
placement), each value timed with the others at their best so far:
`gemm_rows_per_thread` (rows per thread of the narrow tall products: 1 keeps
more warps resident, 2 halves the shared-memory reads per multiply-add) and
`dst_cta_threads` (columns of the shared-memory DST per CTA).  Neither changes
an operation or its order: single plans return the same bits under every value
(a GPU test).  The tuner checks this for every candidate on a single plan
(one lane) of the first problems, bit for bit, and refuses the candidate
otherwise; the timing runs use the chosen lanes, where the results of
concurrent lanes have been seen to part in rare problems (the largest relative
difference of the low-rank products between the candidates' timing runs is
recorded).

    python -m paper_2607_06021_gb300.tune --write TABLE.json

tunes the bench workload (n = 4095, rank-20 right-hand sides, tol 1e-8, rank
cap 64, index capacity 64; both precisions, batches of 256 and 1024) on the
current GPU and writes the table.
"""
from __future__ import annotations

import json
import os
import statistics
from typing import Callable, Dict, Iterable, List, Optional, Tuple

DEFAULT_LANES = (1, 2, 4, 8)
# (lanes, loop on the device)
DEFAULT_CONFIGS = ((1, False), (2, False), (4, False), (8, False), (1, True), (2, True), (4, True))
TIE = 0.01  # candidates within 1% of the fastest count as ties
# result-neutral launch shapes (lrp_opts fields), values in order of preference on ties
SHAPE_KNOBS = (("gemm_rows_per_thread", (2, 1)), ("dst_cta_threads", (256, 512, 1024)))
DEFAULT_SHAPES = {"gemm_rows_per_thread": 0, "dst_cta_threads": 0}
TABLE_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_gb300.json")


def rank_class(r_f: int) -> int:
    """Right-hand-side rank bucket: the smallest power of two >= r_f (>= 1)."""
    c = 1
    while c < max(1, int(r_f)):
        c <<= 1
    return c


def table_key(precision: str, n: int, r_f: int, batch: int) -> str:
    return f"{precision}/n{int(n)}/rf{rank_class(r_f)}/b{int(batch)}"


def config_name(cfg) -> str:
    """'4' for 4 lanes with host loops, '4d' with device loops (a bare int is host loops)."""
    lanes, dev = (cfg, False) if isinstance(cfg, int) else cfg
    return f"{int(lanes)}{'d' if dev else ''}"


def candidate_lanes(batch: int, candidates: Iterable[int] = DEFAULT_LANES) -> List[int]:
    """Lane counts worth timing: every lane gets at least one problem."""
    return sorted({int(c) for c in candidates if 1 <= int(c) <= int(batch)})


def candidate_configs(batch: int, candidates=DEFAULT_CONFIGS) -> List[Tuple[int, bool]]:
    """(lanes, device loop) configurations worth timing: every lane gets a problem."""
    return sorted({(int(l), bool(d)) for l, d in candidates if 1 <= int(l) <= int(batch)})


def choose(times: Dict) -> object:
    """The configuration with the smallest median time; candidates within TIE
    of it count as ties, which go to the smallest configuration (fewest lanes,
    then host loops: less memory, fewer streams)."""
    med = {c: statistics.median(ts) for c, ts in times.items() if ts}
    if not med:
        raise ValueError("no timed candidate")
    best = min(med.values())
    return min(c for c, m in med.items() if m <= best * (1.0 + TIE))


def tune_lanes(measure: Callable[[int], List[float]], batch: int,
               candidates: Iterable[int] = DEFAULT_LANES) -> Tuple[int, Dict[int, List[float]]]:
    """measure(lanes) -> timed runs (ms) of one batch at that lane count;
    returns the chosen lane count and every candidate's times."""
    times = {lanes: list(measure(lanes)) for lanes in candidate_lanes(batch, candidates)}
    return choose(times), times


def tune_configs(measure: Callable[[Tuple[int, bool]], List[float]], batch: int, candidates=DEFAULT_CONFIGS):
    """measure((lanes, device_loop)) -> timed runs (ms); returns the chosen
    configuration and every candidate's times."""
    times = {cfg: list(measure(cfg)) for cfg in candidate_configs(batch, candidates)}
    return choose(times), times


def choose_first(times: Dict, order) -> object:
    """The fastest value by median; values within TIE of it count as ties, which
    go to the earliest value in `order`."""
    med = {c: statistics.median(ts) for c, ts in times.items() if ts}
    if not med:
        raise ValueError("no timed candidate")
    best = min(med.values())
    return next(c for c in order if c in med and med[c] <= best * (1.0 + TIE))


def tune_shapes(measure: Callable[[Dict[str, int]], List[float]], knobs=SHAPE_KNOBS):
    """Coordinate descent over the launch shapes: for each knob in turn, time
    every value with the other knobs at their best so far (starting from the
    first listed value of each); measure(shapes) -> timed runs (ms).  Returns the
    chosen shapes and {knob: {value: [ms]}}."""
    best = {name: values[0] for name, values in knobs}
    times: Dict[str, Dict[int, List[float]]] = {}
    for name, values in knobs:
        t = {}
        for v in values:
            t[v] = list(measure(dict(best, **{name: v})))
        best[name] = choose_first(t, values)
        times[name] = t
    return best, times


class TuneTable:
    """Chosen configurations, persisted as JSON
    ({key: {"lanes": L, "loop_on_device": bool, "ms": {name: median}}})."""

    def __init__(self, path: Optional[str] = None):
        self.path = path
        self.entries: Dict[str, dict] = {}
        if path and os.path.exists(path):
            with open(path) as f:
                self.entries = json.load(f)

    def get_config(self, precision: str, n: int, r_f: int, batch: int) -> Optional[Tuple[int, bool]]:
        e = self.entries.get(table_key(precision, n, r_f, batch))
        return (int(e["lanes"]), bool(e.get("loop_on_device", False))) if e else None

    def get_shapes(self, precision: str, n: int, r_f: int, batch: int) -> Dict[str, int]:
        """The tuned launch shapes (lrp_opts fields; 0 = the library default)."""
        e = self.entries.get(table_key(precision, n, r_f, batch)) or {}
        return {k: int(e.get(k, DEFAULT_SHAPES[k])) for k in DEFAULT_SHAPES}

    def get(self, precision: str, n: int, r_f: int, batch: int) -> Optional[int]:
        c = self.get_config(precision, n, r_f, batch)
        return c[0] if c else None

    def put(self, precision: str, n: int, r_f: int, batch: int, cfg, times: Dict, extra: Optional[dict] = None):
        lanes, dev = (cfg, False) if isinstance(cfg, int) else cfg
        e = {"lanes": int(lanes), "ms": {config_name(k): statistics.median(v) for k, v in times.items() if v}}
        if dev or not isinstance(cfg, int):
            e["loop_on_device"] = bool(dev)
        if extra:
            e.update(extra)
        self.entries[table_key(precision, n, r_f, batch)] = e

    def save(self) -> None:
        if not self.path:
            return
        tmp = self.path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(self.entries, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


def autotune_group(n: int, tol: float, max_rank: int, inputs, precision: str = "mixed",
                   candidates=DEFAULT_CONFIGS, reps: int = 3,
                   table: Optional[TuneTable] = None, stream=None, extra: Optional[dict] = None, **group_kw):
    """(lanes, device_loop) for solving `inputs` (a list of (U_f, s_f, V_f)
    device tensors, one problem each) with lrp_group.  A table hit returns at
    once; otherwise each candidate gets its own group (created, warmed up, timed
    `reps` times, closed before the next, so that only one workspace is held)
    and the choice is recorded in the table.  Candidates are (lanes, device
    loop) pairs or bare lane counts (host loops).  Returns (config, {config: [ms]})."""
    import torch

    from .api import Group
    batch = len(inputs)
    r_f = max(int(U.shape[1]) for U, _, _ in inputs)
    if table is not None:
        hit = table.get_config(precision, n, r_f, batch)
        if hit is not None:
            return hit, {}
    s = torch.cuda.current_stream() if stream is None else stream
    cands = [(c, False) if isinstance(c, int) else tuple(c) for c in candidates]

    def measure(cfg) -> List[float]:
        lanes, dev = cfg
        g = Group(n, tol, max_rank, lanes=lanes, precision=precision, batch=batch, max_rhs_rank=r_f,
                  loop_on_device=dev, **group_kw)
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

    cfg, times = tune_configs(measure, batch, cands)
    if table is not None:
        table.put(precision, n, r_f, batch, cfg, times, extra)
        table.save()
    return cfg, times


def autotune_shapes(n: int, tol: float, max_rank: int, inputs, cfg, precision: str = "mixed", reps: int = 3,
                    stream=None, knobs=SHAPE_KNOBS, check: int = 64, **group_kw):
    """The launch shapes for `inputs` at the (lanes, device loop) configuration
    `cfg`, by tune_shapes.  Each candidate first solves the first `check`
    problems on a single plan; its results must equal the first candidate's bit
    for bit (rank columns of U, V, rank values of S, the info record), else
    RuntimeError.  Returns (shapes, {knob: {value: [ms]}}, the largest relative
    difference of the low-rank products between the timing runs' results)."""
    import torch

    from .api import Group, Plan, parse_info
    batch = len(inputs)
    r_f = max(int(U.shape[1]) for U, _, _ in inputs)
    s = torch.cuda.current_stream() if stream is None else stream
    lanes, dev = (cfg, False) if isinstance(cfg, int) else cfg
    ref_plan, ref = [], []
    worst = [0.0]
    sub = inputs[:max(1, min(check, batch))]

    def defined(outs):
        # rank columns of U and V, rank values of S, the info record (columns
        # past the rank are unspecified)
        res = []
        for U, S, V, info in outs:
            r = int(parse_info(info)["rank"])
            res.append((U[:, :r].clone(), S[:r].clone(), V[:, :r].clone(), info.clone()))
        return res

    def measure(shapes) -> List[float]:
        p = Plan(n, tol, max_rank, precision=precision, batch=len(sub), max_rhs_rank=r_f, **shapes, **group_kw)
        try:
            outs = [p.alloc_outputs() for _ in sub]
            p.solve_batch_into(sub, outs, s)
            torch.cuda.synchronize()
            res = defined(outs)
        finally:
            p.close()
        if not ref_plan:
            ref_plan.extend(res)
        elif not all(x.shape == y.shape and torch.equal(x, y) for a, b in zip(ref_plan, res) for x, y in zip(a, b)):
            raise RuntimeError(f"launch shapes {shapes} changed a single plan's results")
        g = Group(n, tol, max_rank, lanes=lanes, precision=precision, batch=batch, max_rhs_rank=r_f,
                  loop_on_device=dev, **shapes, **group_kw)
        try:
            outs = [g.alloc_outputs() for _ in inputs]
            g.solve_batch_into(inputs, outs, s)
            torch.cuda.synchronize()
            res = [x[:3] for x in defined(outs)]
            if not ref:
                ref.extend(res)
            else:
                for a, b in zip(ref, res):
                    worst[0] = max(worst[0], lowrank_rel_diff(a, b))
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

    shapes, times = tune_shapes(measure, knobs)
    return shapes, times, worst[0]


def lowrank_rel_diff(a, b) -> float:
    """||U S V^T - U' S' V'^T||_F / ||U S V^T||_F of two results (U, S, V)
    without forming the n x n products: Gram identity on the small factors."""
    import torch
    if all(x.shape == y.shape and torch.equal(x, y) for x, y in zip(a, b)):
        return 0.0
    U, S, V = (t.double() for t in a)
    U2, S2, V2 = (t.double() for t in b)
    aa = float((S * S).sum()) if S.numel() else 0.0
    bb = float((S2 * S2).sum()) if S2.numel() else 0.0
    ab = float(((S[:, None] * (U.T @ U2)) * ((V.T @ V2) * S2[None, :])).sum()) if S.numel() and S2.numel() else 0.0
    return (max(aa + bb - 2.0 * ab, 0.0) ** 0.5) / max(aa ** 0.5, 1e-300)


def _main():
    import argparse
    import sys
    import time

    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--write", default=TABLE_PATH)
    ap.add_argument("--batches", default="256,1024")
    a = ap.parse_args()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import lrp_inputs as li

    def dev(x):
        import numpy as np
        x = np.asarray(x, dtype=np.float64)
        return torch.from_numpy(x.copy()).cuda() if x.ndim == 1 else torch.from_numpy(np.ascontiguousarray(x.T)).cuda().t()

    table = TuneTable(a.write)
    gpu = torch.cuda.get_device_name(0)
    for B in [int(b) for b in a.batches.split(",")]:
        rhss = [li.workload_n4095(seed=s) for s in range(B)]
        inputs = [(dev(r.U), dev(r.s), dev(r.V)) for r in rhss]
        for prec in ("mixed", "fp64"):
            t0 = time.time()
            cfg, times = autotune_group(4095, 1e-8, 64, inputs, precision=prec, table=None, m_cap=64,
                                        max_iter=30)
            shapes, stimes, worst = autotune_shapes(4095, 1e-8, 64, inputs, cfg, precision=prec, m_cap=64,
                                                    max_iter=30)
            extra = {"gpu": gpu, "tuned_s": round(time.time() - t0, 1), "shapes_max_rel_diff": worst,
                     "shape_ms": {k: {str(v): round(statistics.median(t), 3) for v, t in tv.items()}
                                  for k, tv in stimes.items()}}
            extra.update(shapes)
            table.put(prec, 4095, 20, B, cfg, times, extra)
            table.save()
            print(prec, B, config_name(cfg), {config_name(k): round(statistics.median(v), 2) for k, v in times.items()},
                  shapes, extra["shape_ms"], flush=True)


if __name__ == "__main__":
    _main()

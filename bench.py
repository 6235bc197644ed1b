#!/usr/bin/env python3
"""Batched low-rank Poisson solves on GB300: solves/s and p50/p99 step latency.

Workload (one "step" = one batch of independent solves through the whole hot
path: forward DST, Cross-DEIM iterations, back DST): n = 4095 interior points
(h = 1/4096), right-hand side of rank 20 (16 seeded separable Gaussians + 4
discrete eigenfunctions with p, q in 1..64), tol 1e-8, max rank 64, seeds
distinct per problem and rank.  Both precisions run side by side; the headline
`value` is the mixed-precision path when it is built, else FP64.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun each rank solves its own batch on its own GPU (replicas, weak
scaling, no data-path collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N = 4095
TOL = 1e-8
RMAX = 64
RF = 20
M_CAP = 64  # index-set capacity; the sets reach at most ~35 on this workload
ERR_CHECK = 256  # problems of the timed batch whose error against the exact solution is checked
ERR_BAR = 1e-6   # the metric's accuracy bar
STATUS_NAMES = {0: "LRP_OK", 5: "LRP_NOT_CONVERGED", 6: "LRP_RANK_CAPPED"}
WORKLOAD = ("n=4095 (h=1/4096), RHS rank 20 = 16 seeded Gaussians + 4 eigenfunctions "
            "(p,q in 1..64), tol 1e-8, max rank 64, index-set capacity 64")
METRIC = "Poisson solves/s & p50/p99 latency at rel err<=1e-6, mixed vs plain FP64"
# ALU peaks from unit counts and the maximum SM clock (152 SMs, 2070 MHz):
# FP64 4 flop/clk/SM (2 FMA), FP32 256 flop/clk/SM (128 lanes x FMA).  Double-
# float arithmetic runs on the FP32 lanes (128 instructions/clk/SM): a multiply-
# add of FP32 data into a (hi, lo) sum takes 10 instructions (exact product by
# FMA, TwoSum, low-part sum), one of (hi, lo) data 13 (plus the cross terms), and
# the FFT's double-float butterflies ~14.8 instructions per nominal flop (an add
# 20, a multiply 7; a radix-2 butterfly 4 multiplies and 6 adds for 10 flops).
SMS, SM_GHZ = 152, 2.070
FP64_PEAK_TFLOPS = SMS * 4 * SM_GHZ / 1e3
FP32_PEAK_TFLOPS = SMS * 256 * SM_GHZ / 1e3
FP32_LANE_TOPS = SMS * 128 * SM_GHZ / 1e3
DF_MADD32_TFLOPS = FP32_LANE_TOPS / 10 * 2
DF_MADD_TFLOPS = FP32_LANE_TOPS / 13 * 2
DF_FFT_TFLOPS = FP32_LANE_TOPS / 14.8
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lrp", choices=["lrp", "reference"])
    ap.add_argument("--batch", type=int, default=1024, help="problems per step (per GPU)")
    ap.add_argument("--lanes", type=int, default=0,
                    help="concurrent sub-batches (lrp_group), 1 = one plan; 0 = the tuned table's choice, else 4")
    ap.add_argument("--loop-on-device", type=int, default=-1,
                    help="1: iteration loops on the device (one graph per solve); -1 = the tuned table's choice")
    ap.add_argument("--precision", default="both", choices=["fp64", "mixed", "both"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--err-check", type=int, default=ERR_CHECK,
                    help="problems of the batch checked against the exact solution (0: all)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--refine-steps", type=int, default=2,
                    help="mixed precision: 1 residual-correction step, or 2 (a second one where the first looks unreliable)")
    ap.add_argument("--selector", default="bernoulli", choices=["ls", "bernoulli", "qdeim"],
                    help="index selector: leverage top-c, leverage Bernoulli sampling, or QDEIM")
    ap.add_argument("--sample-factor", type=float, default=1.0, help="Bernoulli c / columns")
    ap.add_argument("--sweep", action="store_true",
                    help="instead of the bench line: solve time, rank and iterations against n (Sec. 4.2 scaling)")
    ap.add_argument("--sweep-kmin", type=int, default=10)
    ap.add_argument("--sweep-kmax", type=int, default=20)
    ap.add_argument("--sweep-seeds", type=int, default=3, help="growth-index seeds per size")
    ap.add_argument("--sweep-selectors", default="bernoulli,ls,qdeim", help="index selectors of the sweep")
    ap.add_argument("--sweep-sample-factor", type=float, default=1.0, help="Bernoulli c / columns in the sweep")
    ap.add_argument("--test-matrices", action="store_true",
                    help="instead of the bench line: Cross-DEIM on the test matrices of Sec. 4.1")
    ap.add_argument("--serve-requests", type=int, default=800,
                    help="requests of the serving stream (0: skip)")
    ap.add_argument("--serve-rate", type=float, default=150.0, help="Poisson arrival rate, requests/s")
    ap.add_argument("--serve-kmax", type=int, default=14, help="largest n = 2^k - 1 of the stream")
    ap.add_argument("--mixed-sizes", type=int, default=512, help="solves of the mixed-size batch (0: skip)")
    ap.add_argument("--serve-sweep", action="store_true",
                    help="instead of the bench line: the serving stream at several offered rates (n up to 2^18-1)")
    ap.add_argument("--serve-sweep-rates", default="1000,2000,5000,10000,20000")
    ap.add_argument("--serve-sweep-requests", type=int, default=4000, help="requests per offered rate")
    ap.add_argument("--serve-sweep-kmax", type=int, default=18)
    ap.add_argument("--serve-lanes", type=int, default=4)
    ap.add_argument("--serve-frac-fp64", type=float, default=0.2, help="share of FP64 requests in the stream")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def replica_barrier(world: int) -> None:
    """Barrier of the replicas (one process per GPU; no-op alone)."""
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def replica_max(v: float, world: int, device) -> float:
    """The largest of the ranks' values (the whole job's timed region)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seeds(rank: int, batch: int) -> list:
    """Input seeds of a rank's batch: disjoint across ranks (weak scaling)."""
    return [1000 * rank + i for i in range(batch)]


def whole_job_value(batch: int, world: int, steps: int, total_ms: float) -> float:
    """Solves per second of all ranks together over the slowest rank's time."""
    return batch * world * steps / (total_ms / 1e3)


def to_dev(a):
    """A host NumPy array as a CUDA float64 tensor (2-D: column-major)."""
    import numpy as np
    import torch
    a = np.asarray(a, dtype=np.float64)
    if a.ndim == 1:
        return torch.from_numpy(a.copy()).cuda()
    return torch.from_numpy(np.ascontiguousarray(a.T)).cuda().t()


def to_np(t):
    import numpy as np
    return t.detach().cpu().numpy().astype(np.float64)


def rhs_dev(rhs):
    """Device copies of a right-hand side's factors (U_f, s_f, V_f)."""
    return to_dev(rhs.U), to_dev(rhs.s), to_dev(rhs.V)


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json)"
    except Exception:
        return 6800.0, "fallback (profiling recipe)"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.file = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.file.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.file.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------- GPU arm

class Batch:
    """Device-resident inputs and outputs of one batch, packed for single H2D / D2H copies."""

    def __init__(self, rhss, torch, device):
        import numpy as np
        self.B = len(rhss)
        per_in = 2 * N * RF + RF
        per_out = 2 * N * RMAX + RMAX + 8
        host_in = np.zeros(self.B * per_in)
        for b, r in enumerate(rhss):
            o = b * per_in
            host_in[o:o + N * RF] = r.U.reshape(-1, order="F")
            host_in[o + N * RF:o + 2 * N * RF] = r.V.reshape(-1, order="F")
            host_in[o + 2 * N * RF:o + per_in] = r.s
        self.host_in = torch.from_numpy(host_in).pin_memory()
        self.dev_in = self.host_in.to(device)
        self.dev_out = torch.zeros(self.B * per_out, dtype=torch.float64, device=device)
        self.host_out = torch.zeros(self.B * per_out, dtype=torch.float64).pin_memory()
        self.inputs, self.outputs = [], []
        for b in range(self.B):
            o = b * per_in
            U = self.dev_in[o:o + N * RF].view(RF, N).t()
            V = self.dev_in[o + N * RF:o + 2 * N * RF].view(RF, N).t()
            s = self.dev_in[o + 2 * N * RF:o + per_in]
            self.inputs.append((U, s, V))
            q = b * per_out
            Uo = self.dev_out[q:q + N * RMAX].view(RMAX, N).t()
            Vo = self.dev_out[q + N * RMAX:q + 2 * N * RMAX].view(RMAX, N).t()
            So = self.dev_out[q + 2 * N * RMAX:q + 2 * N * RMAX + RMAX]
            info = self.dev_out[q + 2 * N * RMAX + RMAX:q + per_out].view(torch.uint8)
            self.outputs.append((Uo, So, Vo, info))
        # End-to-end pipeline: a second input slot, two compact result buffers
        # (lrp_plan_pack: rank columns only) and two host destinations.
        self.dev_in2 = torch.empty_like(self.dev_in)
        self.inputs2 = []
        for b in range(self.B):
            o = b * per_in
            self.inputs2.append((self.dev_in2[o:o + N * RF].view(RF, N).t(),
                                 self.dev_in2[o + 2 * N * RF:o + per_in],
                                 self.dev_in2[o + N * RF:o + 2 * N * RF].view(RF, N).t()))
        self.packed = [torch.zeros(self.B * per_out, dtype=torch.float64, device=device) for _ in range(2)]
        self.offsets = [torch.zeros(self.B + 1, dtype=torch.int64, device=device) for _ in range(2)]
        self.host_res = [self.host_out, torch.zeros(self.B * per_out, dtype=torch.float64).pin_memory()]
        self.h2d_bytes = self.host_in.numel() * 8


def time_steps(fn, K, stream, torch, flush):
    evs = []
    for _ in range(K):
        flush.zero_()  # L2 flush: 256 MiB write between timed steps
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def e2e_pipeline(plan, batch, stream, K, torch):
    """K steps through the public API with host buffers: each step's inputs go
    host -> device (pinned) and its compact results device -> host, all inside
    the timed region; copies run on a second stream, double-buffered, so that the
    next step's inputs and the previous step's results move while a step solves."""
    B = batch.B
    copy = torch.cuda.Stream(device=stream.device)
    ev = lambda: torch.cuda.Event()  # noqa: E731
    in_ready, done, out_done = [ev(), ev()], [ev(), ev()], [ev(), ev()]
    dev_in, inputs = [batch.dev_in, batch.dev_in2], [batch.inputs, batch.inputs2]
    d2h = []
    torch.cuda.synchronize()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    copy.wait_event(start)
    with torch.cuda.stream(copy):
        dev_in[0].copy_(batch.host_in, non_blocking=True)
        in_ready[0].record(copy)
    def fetch(j):
        # results of step j (already packed) move to the host on the copy stream;
        # reading their size waits only for step j, not for the step queued after it
        sj = j & 1
        total = int(batch.offsets[sj][B].item())
        with torch.cuda.stream(copy):
            copy.wait_event(done[sj])
            batch.host_res[sj][:total].copy_(batch.packed[sj][:total], non_blocking=True)
            out_done[sj].record(copy)
        d2h.append(8 * (total + B + 1))

    for k in range(K):
        s = k & 1
        # the next step's inputs move while this step solves (slot 1-s was last
        # read by step k-1)
        if k + 1 < K:
            with torch.cuda.stream(copy):
                if k >= 1:
                    copy.wait_event(done[1 - s])
                dev_in[1 - s].copy_(batch.host_in, non_blocking=True)
                in_ready[1 - s].record(copy)
        with torch.cuda.stream(stream):
            stream.wait_event(in_ready[s])
            plan.solve_batch_into(inputs[s], batch.outputs, stream)
            if k >= 2:
                stream.wait_event(out_done[s])  # packed[s] of step k-2 has been read
            plan.pack(batch.packed[s], batch.offsets[s], stream)
            done[s].record(stream)
        if k >= 1:
            fetch(k - 1)
    fetch(K - 1)
    stream.wait_stream(copy)
    end.record(stream)
    torch.cuda.synchronize()
    return start.elapsed_time(end), d2h


def copy_bandwidth(batch, stream, torch):
    """GB/s of one host-to-device copy of a step's inputs and one device-to-host
    copy of the same number of bytes of packed results (pinned host memory)."""
    out = {}
    n_in = batch.host_in.numel() * batch.host_in.element_size()
    n_out = min(batch.packed[0].numel(), batch.host_res[0].numel())
    for name, fn, nbytes in (("h2d_gbs", lambda: batch.dev_in.copy_(batch.host_in, non_blocking=True), n_in),
                             ("d2h_gbs", lambda: batch.host_res[0][:n_out].copy_(batch.packed[0][:n_out],
                                                                                non_blocking=True), 8 * n_out)):
        with torch.cuda.stream(stream):
            fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
        out[name] = round(nbytes / (e0.elapsed_time(e1) / 1e3) / 1e9, 1)
    return out


def gpu_arm(args, rank, world, local_rank, precisions):
    import torch

    import lrp_inputs as li
    import paper_2607_06021_gb300 as lrp

    torch.cuda.set_device(local_rank)
    device = torch.device("cuda", local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=device)
    B = args.batch
    rhss = [li.workload_n4095(seed=sd) for sd in replica_seeds(rank, B)]
    batch = Batch(rhss, torch, device)
    stream = torch.cuda.Stream(device=device)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)
    hbm_peak, peak_src = load_peaks()

    def barrier():
        replica_barrier(world)

    def max_over_ranks(v: float) -> float:
        return replica_max(v, world, device)

    results = {}
    from paper_2607_06021_gb300 import tune
    table = tune.TuneTable(tune.TABLE_PATH)
    for prec in precisions:
        # lanes and loop placement: the command line, else the tuned table (both
        # leave the results unchanged), else 4 lanes with host loops
        cfg = table.get_config(prec, N, RF, B)
        lanes = args.lanes if args.lanes > 0 else (cfg[0] if cfg else 4)
        dev = bool(args.loop_on_device) if args.loop_on_device >= 0 else (cfg[1] if cfg else False)
        src = "table" if (cfg and args.lanes <= 0 and args.loop_on_device < 0) else "command line / default"
        # launch shapes: the tuned table's (result-neutral; 0 = library default)
        shapes = table.get_shapes(prec, N, RF, B)
        if lanes > 1:
            plan = lrp.Group(N, TOL, RMAX, lanes=lanes, precision=prec, batch=B, max_rhs_rank=RF, m_cap=M_CAP,
                             refine_steps=args.refine_steps, selector=args.selector,
                             sample_factor=args.sample_factor, loop_on_device=dev, **shapes)
        else:
            plan = lrp.Plan(N, TOL, RMAX, precision=prec, batch=B, max_rhs_rank=RF, m_cap=M_CAP,
                            refine_steps=args.refine_steps, selector=args.selector, sample_factor=args.sample_factor,
                            loop_on_device=dev, **shapes)

        def step():
            with torch.cuda.stream(stream):
                plan.solve_batch_into(batch.inputs, batch.outputs, stream)

        # The clock sampler starts before the warm-up steps: its start-up (NVML
        # initialisation) stays out of the timed region; it samples through it.
        clocks = ClockSampler(local_rank)
        clocks.start()
        time.sleep(0.5)
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                step()
        torch.cuda.synchronize()
        plan.reset_stats()
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            ms = time_steps(step, args.steps, stream, torch, flush)
        wall = time.perf_counter() - t0
        clk = clocks.stop()
        torch.cuda.synchronize()
        barrier()
        launches = plan.kernel_stats()["all"][0]
        total_ms = max_over_ranks(sum(ms))
        res = {"ms": ms, "total_ms": total_ms, "wall_s": wall, "clocks": clk, "launches": launches,
               "value": whole_job_value(B, world, args.steps, total_ms),
               "tuning": {"lanes": lanes, "loop_on_device": dev, "source": src, **shapes}}
        # End to end through the public call with host buffers (pinned), copies inside the timed region.
        if not args.no_e2e:
            barrier()
            e2e_total, d2h = e2e_pipeline(plan, batch, stream, args.steps, torch)
            e2e_total = max_over_ranks(e2e_total)
            res["e2e"] = {"value": whole_job_value(B, world, args.steps, e2e_total), "unit": "solves/s",
                          "h2d_bytes_per_step": batch.h2d_bytes,
                          "d2h_bytes_per_step": int(sum(d2h) / max(len(d2h), 1)),
                          "results": "compact: rank columns of U, V and rank values of S per problem (lrp_plan_pack)",
                          "pipeline": "next step's H2D and previous step's D2H on a copy stream, overlapping the solve"}
            res["e2e"].update(copy_bandwidth(batch, stream, torch))
        # Per-problem reports of the last step.
        torch.cuda.synchronize()
        infos = [lrp.parse_info(o[3]) for o in batch.outputs]
        res["infos"] = infos
        res["results"] = [(o[0].cpu().numpy(), o[1].cpu().numpy(), o[2].cpu().numpy()) for o in batch.outputs]
        plan.close()
        # Per-kernel-class event timing and algorithmic work: a separate pass on
        # one plan of the same batch, so that no launch shares the GPU with
        # another lane's (concurrent lanes would fold their waits into each
        # launch's event interval).
        tplan = lrp.Plan(N, TOL, RMAX, precision=prec, batch=B, max_rhs_rank=RF, m_cap=M_CAP,
                         refine_steps=args.refine_steps, selector=args.selector, sample_factor=args.sample_factor,
                         **shapes)
        with torch.cuda.stream(stream):
            tplan.solve_batch_into(batch.inputs, batch.outputs, stream)
        tplan.set_timing(True)
        tplan.reset_stats()
        with torch.cuda.stream(stream):
            time_steps(lambda: tplan.solve_batch_into(batch.inputs, batch.outputs, stream), 2, stream, torch, flush)
        res["kernels"] = tplan.kernel_stats()
        tplan.set_timing(False)
        tplan.close()
        results[prec] = res
    return results, rhss, hbm_peak, peak_src


# The arithmetic pipe of each kernel class with algorithmic flops; every class is
# held to the roofline max(flops / pipe peak, bytes / HBM peak), its bound the
# larger term.  FP64 path: every product and the DST on the FP64 pipe.  Mixed
# path: the FP32 iterations on the FP32 pipe, the double-float Grams, products
# and DST on the FP32 lanes at their instruction counts.
PIPES = {"fp64": {"gram": "fp64", "gemm": "fp64", "cross": "fp64", "reduce": "fp64", "dst": "fp64",
                  "leverage": "fp64"},
         "mixed": {"gram_f32": "fp32", "gemm_f32": "fp32", "cross": "fp32", "dst": "fp32", "leverage": "fp32",
                   "reduce": "fp64", "gram_df": "df32", "gemm_df": "df", "dst_df": "df_fft",
                   "gram": "fp64", "gemm": "fp64"}}
ALU_PEAKS = {"fp64": FP64_PEAK_TFLOPS, "fp32": FP32_PEAK_TFLOPS, "df32": DF_MADD32_TFLOPS,
             "df": DF_MADD_TFLOPS, "df_fft": DF_FFT_TFLOPS}
PEAK_SOURCE = {"fp64": "FP64 pipe: 152 SMs x 2070 MHz x 4 flop/clk/SM",
               "fp32": "FP32 pipe: 152 SMs x 2070 MHz x 256 flop/clk/SM",
               "df32": "double-float multiply-add of FP32 data: 152 SMs x 2070 MHz x 128 lanes / 10 instructions x 2 flop",
               "df": "double-float multiply-add of (hi, lo) data: 152 SMs x 2070 MHz x 128 lanes / 13 instructions x 2 flop",
               "df_fft": "double-float FFT: 152 SMs x 2070 MHz x 128 lanes / 14.8 instructions per flop"}
# DRAM bytes (read + write) per launch from ncu captures of the mixed bench at
# batch 128, scaled by batch / 128 (the launches' data grow with the slots);
# a class whose kernel changed since its capture has no entry.
TRAFFIC_B128 = {("mixed", "gram_df"): (87.0e6, "profiles/k_gram_df_mixed_n4095_batch128.md")}


def class_bound(prec, name, launches, ms, flops, nbytes, hbm_peak):
    """Roofline of one kernel class: the larger of its ALU and HBM times."""
    t = ms / 1e3
    pipe = PIPES[prec].get(name)
    t_alu = flops / (ALU_PEAKS[pipe] * 1e12) if pipe else 0.0
    t_hbm = nbytes / (hbm_peak * 1e9)
    if pipe and t_alu >= t_hbm:
        achieved = flops / t / 1e12
        return {"bound": "alu", "pipe": pipe, "achieved": achieved, "peak": ALU_PEAKS[pipe], "unit": "TFLOP/s",
                "frac": achieved / ALU_PEAKS[pipe], "algorithmic_per_launch": flops / launches}
    achieved = nbytes / t / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
            "algorithmic_per_launch": nbytes / launches}


def roofline(res, prec, hbm_peak, peak_src, batch):
    """Dominant kernel class (most event-timed time, among classes with
    algorithmic work) against its roofline."""
    ks = {k: v for k, v in res["kernels"].items() if k != "all" and v[2] + v[3] > 0}
    if not ks:
        return None
    name = max(ks, key=lambda k: ks[k][1])
    launches, ms, flops, nbytes = ks[name]
    if ms <= 0 or launches <= 0:
        return None
    out = class_bound(prec, name, launches, ms, flops, nbytes, hbm_peak)
    out["peak_source"] = PEAK_SOURCE[out["pipe"]] if out["bound"] == "alu" else peak_src
    out.update({"kernel": name, "launches": launches, "avg_launch_us": 1e3 * ms / launches, "traffic": None})
    tr = TRAFFIC_B128.get((prec, name))
    if tr is not None:
        out["traffic"] = tr[0] * batch / 128
        out["traffic_source"] = (f"{tr[1]} (dram bytes of a launch with every problem active at batch 128, scaled to "
                                 f"batch {batch}; the timed average launch includes later iterations with fewer active)")
    return out


def class_rooflines(res, prec, hbm_peak):
    """Every kernel class with algorithmic work, against its own roofline."""
    out = {}
    for name, (launches, ms, flops, nbytes) in res["kernels"].items():
        if name == "all" or ms <= 0 or flops + nbytes <= 0:
            continue
        b = class_bound(prec, name, launches, ms, flops, nbytes, hbm_peak)
        out[name] = {"bound": b["bound"] if b["bound"] == "hbm" else "alu_" + b["pipe"], "ms": round(ms, 3),
                     "frac": round(b["frac"], 4)}
    return out


def serving_stream(args, rank, rate=None, requests=None, kmax=None, lanes=2, cap_gb=40, keep=32):
    """Poisson arrivals of independent requests through the request server:
    n = 2^k - 1 with k uniform in 8..kmax, r_f uniform in 2..48 Gaussians, 80%
    mixed precision at tol 1e-6 and 20% FP64 at tol 1e-10 (rank cap 64), 10% of
    requests perturbed repeats of an earlier one that reuse its warm-start key.
    Latency runs from the request's arrival time to its completion.  Returns the
    record and up to `keep` served results with n <= 4095 (for the accuracy
    check of the CPU leg)."""
    import numpy as np

    import lrp_inputs as li
    import paper_2607_06021_gb300 as lrp
    rate = args.serve_rate if rate is None else rate
    R = args.serve_requests if requests is None else requests
    kmax = args.serve_kmax if kmax is None else kmax
    rng = np.random.default_rng(7 + rank)
    specs = []
    for i in range(R):
        if i > 0 and rng.random() < 0.10:
            j = int(rng.integers(0, i))
            while specs[j]["repeat_of"] >= 0:
                j = specs[j]["repeat_of"]
            specs[j]["warm_key"] = j + 1
            s = dict(specs[j], repeat_of=j, warm_key=j + 1, pert=int(rng.integers(1 << 30)))
        else:
            k = int(rng.integers(8, kmax + 1))
            mixed = rng.random() >= args.serve_frac_fp64
            s = {"n": (1 << k) - 1, "r_f": int(rng.integers(2, 49)), "seed": int(rng.integers(1 << 30)),
                 "prec": "mixed" if mixed else "fp64", "tol": 1e-6 if mixed else 1e-10, "repeat_of": -1,
                 "warm_key": 0, "pert": 0}
        specs.append(s)
    rhss = []
    for s in specs:
        base = li.gaussian_eigen_rhs(s["n"], s["seed"], s["r_f"])
        rhss.append(li.perturb_amplitudes(base, s["pert"]) if s["repeat_of"] >= 0 else base)
    gaps = rng.exponential(1.0 / rate, size=R)
    arrivals = np.cumsum(gaps)
    sv = lrp.Server(memory_cap_bytes=int(cap_gb) << 30, lanes=lanes, max_batch=32, warm_capacity=64)
    # warm the server's plans on one request per bucket (untimed)
    seen = set()
    for s, r in zip(specs, rhss):
        key = (s["n"], s["prec"], (s["r_f"] + 15) // 16)
        if key in seen:
            continue
        seen.add(key)
        sv.wait(sv.submit(r.U, r.s, r.V, s["tol"], 64, s["prec"]), 600.0)
    sv.reset_stats()
    tickets = [None] * R
    delay_us = np.zeros(R)
    t0 = time.perf_counter()
    for i, (s, r) in enumerate(zip(specs, rhss)):
        now = time.perf_counter() - t0
        if arrivals[i] > now:
            time.sleep(arrivals[i] - now)
        while True:
            t = sv.submit(r.U, r.s, r.V, s["tol"], 64, s["prec"], warm_key=s["warm_key"])
            if t is not None:
                break
            time.sleep(1e-4)  # server full: retry
        tickets[i] = t
        delay_us[i] = max(0.0, (time.perf_counter() - t0 - arrivals[i]) * 1e6)
    lat, warm_hits, statuses, by_class = np.zeros(R), 0, {}, {}
    service = {}  # per class: batch start to completion (ms), and time queued (ms)
    kept = []
    for i, t in enumerate(tickets):
        res = sv.wait(t, 600.0)
        info = res[3]
        lat[i] = info["latency_us"] + delay_us[i]
        sc = service.setdefault(f"n={specs[i]['n']},{specs[i]['prec']}", [[], []])
        sc[0].append((info["latency_us"] - info["queue_us"]) / 1e3)
        sc[1].append((info["queue_us"] + delay_us[i]) / 1e3)
        warm_hits += info["warm_used"]
        statuses[info["status"]] = statuses.get(info["status"], 0) + 1
        cls = f"n={specs[i]['n']},{specs[i]['prec']}"
        c = by_class.setdefault(cls, {})
        nm = lrp.status_string(info["status"])
        c[nm] = c.get(nm, 0) + 1
        if len(kept) < keep and specs[i]["n"] <= 4095 and i % 3 == 0:
            kept.append((rhss[i], specs[i]["prec"], specs[i]["tol"], res[0], res[1], res[2]))
    wall = time.perf_counter() - t0
    st = sv.stats()
    last_error = sv.last_error()
    sv.close()
    failed = sum(v for k, v in statuses.items() if k not in (lrp.LRP_OK, lrp.LRP_NOT_CONVERGED, lrp.LRP_RANK_CAPPED))
    rec = {"requests": R, "rate_per_s": rate, "wall_s": round(wall, 3), "failed": failed,
           "last_error": last_error or None,
           "throughput_solves_per_s": R / wall,
           "p50_ms": float(np.percentile(lat, 50)) / 1e3, "p99_ms": float(np.percentile(lat, 99)) / 1e3,
           "mean_ms": float(lat.mean()) / 1e3, "rejected_submits": st["rejected"], "warm_hits": warm_hits,
           "status_counts": {lrp.status_string(k): v for k, v in statuses.items()},
           "status_by_class": by_class,
           "time_by_class_ms": {k: {"requests": len(v[0]), "service_mean": round(float(np.mean(v[0])), 2),
                                    "service_total": round(float(np.sum(v[0])), 1),
                                    "queue_mean": round(float(np.mean(v[1])), 2)}
                                for k, v in sorted(service.items())},
           "lanes": lanes, "memory_cap_gb": cap_gb,
           "workload": f"n=2^k-1, k~U{{8..{kmax}}}, r_f~U{{2..48}} Gaussians, "
                       f"{100 * (1 - args.serve_frac_fp64):.0f}% mixed/1e-6, {100 * args.serve_frac_fp64:.0f}% FP64/1e-10, "
                       "rank cap 64, 10% perturbed repeats (warm keys), Poisson arrivals; "
                       "latency from arrival to completion, plans warmed per bucket beforehand"}
    return rec, kept


def _served_error_job(job):
    """Exact relative error of one served result (pool worker)."""
    from oracle import poisson as po
    rhs, U, S, V = job
    return po.rel_error_vs_exact(U, S, V, po.SpectralSolution(rhs.U, rhs.s, rhs.V))


def check_served(kept, pool, sample="every third served request with n <= 4095, exact sums"):
    """Exact errors of a sample of results against the oracle (CPU leg)."""
    import numpy as np
    if not kept:
        return None
    jobs = [(r, U, S, V) for r, _, _, U, S, V in kept]
    e = np.array(pool.map(_served_error_job, jobs) if pool else [_served_error_job(j) for j in jobs])
    bars = np.array([max(10 * tol, 1e-6) if prec == "mixed" else 10 * tol for _, prec, tol, *_ in kept])
    return {"checked": len(kept), "max": float(e.max()), "median": float(np.median(e)),
            "above_bar": int((e > bars).sum()), "bar": "max(10 tol, 1e-6) mixed, 10 tol FP64",
            "sample": sample}


def mixed_sizes_batch(args, rank):
    """One batch of independent solves of mixed sizes through the request server:
    n uniform over {511, 1023, 2047, 4095, 8191}, r_f uniform in 2..24
    Gaussians, mixed precision at tol 1e-6, all submitted at once."""
    import numpy as np

    import lrp_inputs as li
    import paper_2607_06021_gb300 as lrp
    rhss = li.batch_mixed_sizes(args.mixed_sizes, seed=11 + rank)
    sv = lrp.Server(lanes=2, max_batch=128)

    def run():
        t0 = time.perf_counter()
        ts = [sv.submit(r.U, r.s, r.V, 1e-6, 64, "mixed") for r in rhss]
        out = [sv.wait(t, 600.0) for t in ts]
        return time.perf_counter() - t0, out

    run()  # plans created and graphs captured (untimed)
    walls = []
    for _ in range(3):
        w, out = run()
        walls.append(w)
    sv.close()
    w = statistics.median(walls)
    ns = sorted({r.n for r in rhss})
    return {"solves": len(rhss), "wall_s": round(w, 4), "solves_per_s": len(rhss) / w,
            "iterations_mean": float(np.mean([o[3]["iterations"] for o in out])),
            "workload": f"n uniform over {ns}, r_f~U{{2..24}} Gaussians, mixed precision, tol 1e-6, rank cap 64; "
                        "host factors in, host factors out, median of 3 runs"}


def _exact_error_job(job):
    """Relative error of one GPU result against the exact solution (pool worker)."""
    from oracle import poisson as po
    seed, U, S, V = job
    import lrp_inputs as li
    r = li.workload_n4095(seed=seed)
    return po.rel_error_vs_exact(U, S, V, po.SpectralSolution(r.U, r.s, r.V))


def start_error_pool():
    """Worker processes for the exact-error check, started (spawn) before any
    GPU work so that no worker is forked from a process holding a CUDA context."""
    import multiprocessing as mp
    return mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1)))


def mixed_sizes_one_launch(args, rank):
    """The same 512 mixed-size solves as one CUDA graph launch (lrp_multi):
    inputs resident on the device, one branch per grid size, the iteration
    loops on the device; time per launch by CUDA events after warm-up."""
    import numpy as np
    import torch

    import lrp_inputs as li
    import paper_2607_06021_gb300 as lrp
    rhss = li.batch_mixed_sizes(args.mixed_sizes, seed=11 + rank)
    sizes = sorted({r.n for r in rhss})
    counts = [sum(1 for r in rhss if r.n == n) for n in sizes]
    multi = lrp.Multi(sizes, counts, 1e-6, 64, precision="mixed", max_rhs_rank=24, m_cap=64,
                      selector=args.selector, sample_factor=args.sample_factor)
    ins = [rhs_dev(r) for r in rhss]
    outs = [multi.alloc_outputs(r.n) for r in rhss]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for _ in range(2):
            multi.solve_batch_into(ins, outs, stream)  # capture, then one replay
    torch.cuda.synchronize()
    ms = []
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        with torch.cuda.stream(stream):
            multi.solve_batch_into(ins, outs, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    infos = [lrp.parse_info(o[3]) for o in outs]
    kept = []
    for b, (r, o, inf) in enumerate(zip(rhss, outs, infos)):
        if r.n <= 4095 and b % 8 == 0:
            rk = inf["rank"]
            kept.append((r, "mixed", 1e-6, to_np(o[0][:, :rk]), to_np(o[1][:rk]), to_np(o[2][:, :rk])))
    multi.close()
    st = {}
    for i in infos:
        nm = STATUS_NAMES.get(i["status"], str(i["status"]))
        st[nm] = st.get(nm, 0) + 1
    t = statistics.median(ms) / 1e3
    return kept, {"solves": len(rhss), "launches_per_batch": 1, "ms": round(1e3 * t, 3), "solves_per_s": len(rhss) / t,
            "iterations_mean": float(np.mean([i["total_iterations"] for i in infos])), "status_counts": st,
            "sizes": dict(zip([str(n) for n in sizes], counts)),
            "workload": "as mixed_sizes_batch, device-resident inputs, one graph launch per batch (lrp_multi), "
                        "median of 5 launches after warm-up"}


def cpu_baseline(rhss, seeds, seconds, gpu_results=None, check=ERR_CHECK, pool=None):
    """The CPU oracle as it stands, on a bounded sample of the same workload;
    and the exact error of `check` of the last step's GPU results (0: all)."""
    import numpy as np

    from oracle import cross_deim as cd
    try:
        from threadpoolctl import threadpool_info
        cores = max([i.get("num_threads", 1) for i in threadpool_info()] + [1])
    except Exception:
        cores = os.cpu_count()
    r = rhss[0]
    cd.poisson_solve(r.U, r.s, r.V, TOL, RMAX, m_cap=M_CAP)  # warm-up (as the paper does)
    t0 = time.perf_counter()
    done = 0
    while time.perf_counter() - t0 < seconds and done < len(rhss):
        r = rhss[done]
        cd.poisson_solve(r.U, r.s, r.V, TOL, RMAX, seed=0, m_cap=M_CAP)
        done += 1
    dt = time.perf_counter() - t0
    out = {"value": done / dt, "unit": "solves/s", "cores": cores, "kind": "oracle",
           "sample": f"{done} of the batch's problems, solved one after another ({dt:.1f} s)"}
    errs = {}
    if gpu_results:
        B = len(rhss)
        k = B if check <= 0 else min(check, B)
        picks = sorted(set(int(b) for b in np.linspace(0, B - 1, k)))
        for prec, res in gpu_results.items():
            jobs = []
            for b in picks:
                rk = res["infos"][b]["rank"]
                U, S, V = res["results"][b]
                jobs.append((seeds[b], np.ascontiguousarray(U[:, :rk]), S[:rk].copy(), np.ascontiguousarray(V[:, :rk])))
            t1 = time.perf_counter()
            e = np.array(pool.map(_exact_error_job, jobs, chunksize=4) if pool else [_exact_error_job(j) for j in jobs])
            st = {}
            for b in range(B):
                nm = STATUS_NAMES.get(res["infos"][b]["status"], str(res["infos"][b]["status"]))
                st[nm] = st.get(nm, 0) + 1
            errs[prec] = {"checked": len(picks), "of": B, "max": float(e.max()), "p90": float(np.quantile(e, 0.9)),
                          "median": float(np.median(e)), "above_1e-6": int((e > 1e-6).sum()),
                          "status_counts": st, "check_s": round(time.perf_counter() - t1, 1)}
    return out, errs


def reference_arm(args, rank):
    """The oracle on the host cores, on the same workload: K steps of a bounded sample."""
    if rank != 0:
        return
    import lrp_inputs as li
    from oracle import cross_deim as cd
    try:
        from threadpoolctl import threadpool_info
        cores = max([i.get("num_threads", 1) for i in threadpool_info()] + [1])
    except Exception:
        cores = os.cpu_count()
    per_step = 2
    rhss = [li.workload_n4095(seed=i) for i in range(per_step * (args.steps + args.warmup))]
    times = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        for r in rhss[k * per_step:(k + 1) * per_step]:
            cd.poisson_solve(r.U, r.s, r.V, TOL, RMAX, m_cap=M_CAP)
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    total = sum(times)
    value = per_step * args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "batch": per_step, "precision": "fp64"},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} solves per step on the host cores"},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def _timed_solve(plan, inputs, torch):
    """One warm-up solve, then the wall time (ms) of one solve with the
    device synchronised on both sides, and its result on the host."""
    plan.solve(*inputs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    U, S, V, info = plan.solve(*inputs)
    torch.cuda.synchronize()
    return 1e3 * (time.perf_counter() - t0), U, S, V, info


def sweep(args):
    """Solve time, final rank and iterations against n = 2^k - 1 (Sec. 4.2,
    Figs. of the Poisson solver's scaling), for the paper's right-hand side (one
    Gaussian, lrp_inputs.paper_gaussian_rhs), tol 1e-6, rank cap 64, mixed and
    FP64 precision, `sweep_seeds` growth-index seeds per size; the error of
    every solve against the exact solution (exact sums up to n = 4095, the
    oracle's stratified row-sample estimate above).  The exponent of time
    against N_DOF = n^2 is fitted over n >= 2^14 - 1."""
    import numpy as np
    import torch

    import lrp_inputs as li
    import paper_2607_06021_gb300 as lrp
    from oracle import poisson as po
    tol, rmax = 1e-6, 64
    rows = []
    for k in range(args.sweep_kmin, args.sweep_kmax + 1):
        n = (1 << k) - 1
        rhs = li.paper_gaussian_rhs(n)
        G = po.SpectralSolution(rhs.U, rhs.s, rhs.V)
        inputs = rhs_dev(rhs)
        for prec, sel in [(p, s) for s in args.sweep_selectors.split(",") for p in ("mixed", "fp64")]:
            t, it, rk, er = [], [], [], []
            for seed in range(args.sweep_seeds):
                plan = lrp.Plan(n, tol, rmax, precision=prec, max_rhs_rank=1, seed=seed, selector=sel,
                                sample_factor=args.sweep_sample_factor)
                ms, U, S, V, info = _timed_solve(plan, inputs, torch)
                plan.close()
                U, S, V = to_np(U), to_np(S), to_np(V)
                e = (po.rel_error_vs_exact(U, S, V, G) if n <= 4095 else po.rel_error_sampled(U, S, V, G)[0])
                t.append(ms)
                it.append(info["total_iterations"])
                rk.append(info["rank"])
                er.append(e)
            rows.append({"n": n, "precision": prec, "selector": sel, "ms_mean": float(np.mean(t)), "ms_std": float(np.std(t)),
                         "iterations_mean": float(np.mean(it)), "iterations_std": float(np.std(it)),
                         "rank_mean": float(np.mean(rk)), "rank_std": float(np.std(rk)), "rel_err_max": float(max(er))})
        torch.cuda.empty_cache()
    fit = {}
    for sel in args.sweep_selectors.split(","):
        for prec in ("mixed", "fp64"):
            pts = [(2.0 * np.log(r["n"]), np.log(r["ms_mean"])) for r in rows
                   if r["precision"] == prec and r["selector"] == sel and r["n"] >= 16383]
            if len(pts) >= 2:
                x, y = np.array(pts).T
                fit[f"{sel}/{prec}"] = {"exponent_vs_ndof": float(np.polyfit(x, y, 1)[0]), "sizes": len(pts)}
    return {"mode": "sweep", "rhs": "exp(-36((x-0.1)^2+(y-0.55)^2)) on [-1,1]^2 (Sec. 4.2, sign read as +)",
            "tol": tol, "max_rank": rmax, "seeds": args.sweep_seeds, "bernoulli_sample_factor": args.sweep_sample_factor,
            "rows": rows, "fit_n_ge_16383": fit,
            "time": "wall time of one solve after a warm-up solve of the same plan, device synchronised"}


def test_matrices(args):
    """Cross-DEIM on the test matrices of Sec. 4.1 (H at tol 1e-9, K at tol
    1e-6) for three sizes and the QDEIM and leverage-score selectors: time per
    solve, iterations, rank, and the relative Frobenius error against the matrix
    (dense up to n = 8192, else from 256 seeded rows)."""
    import numpy as np
    import torch

    import lrp_inputs as li
    import paper_2607_06021_gb300 as lrp
    from oracle import matrices as om
    out = []
    for kind, tol in (("hilbert", 1e-9), ("k", 1e-6)):
        for n in (1024, 8192, 65536):
            x0 = li.initial_bases(n, 4, 7)
            inputs = rhs_dev(x0)
            G = om.MATRICES[kind](n)
            for sel in ("qdeim", "ls"):
                plan = lrp.Plan(n, tol, 128, max_rhs_rank=4, selector=sel, seed=7, matrix=kind)
                ms, U, S, V, info = _timed_solve(plan, inputs, torch)
                plan.close()
                U, S, V = to_np(U), to_np(S), to_np(V)
                rows = np.arange(n) if n <= 8192 else np.sort(np.random.default_rng(3).choice(n, 256, replace=False))
                A = G.rows(rows)
                err = float(np.linalg.norm(A - (U[rows] * S) @ V.T) / np.linalg.norm(A))
                out.append({"matrix": kind, "n": n, "tol": tol, "selector": sel, "ms": ms,
                            "iterations": info["iterations"], "rank": info["rank"], "status": info["status"],
                            "rel_err": err, "error_rows": "all" if n <= 8192 else 256})
    return {"mode": "test_matrices", "rows": out,
            "time": "wall time of one solve after a warm-up solve of the same plan, device synchronised"}


def main():
    args = parse()
    rank, world, local_rank = dist_env()
    if args.impl == "reference":
        reference_arm(args, rank)
        return
    import paper_2607_06021_gb300 as lrp  # noqa: F401  (fails loudly without the library)
    if args.sweep or args.test_matrices:
        if rank == 0:
            print(json.dumps(sweep(args) if args.sweep else test_matrices(args)))
        return
    if args.serve_sweep:
        if rank == 0:
            rows = []
            for rate in [float(v) for v in args.serve_sweep_rates.split(",")]:
                rec, _ = serving_stream(args, rank, rate=rate, requests=args.serve_sweep_requests,
                                        kmax=args.serve_sweep_kmax, lanes=args.serve_lanes, cap_gb=40)
                rows.append(rec)
            print(json.dumps({"mode": "serving_sweep", "rates": rows}))
        return
    if args.precision == "both":
        precisions = ["fp64", "mixed"]
    else:
        precisions = [args.precision]
    pool = start_error_pool() if (rank == 0 and world == 1 and not args.no_cpu) else None
    results, rhss, hbm_peak, peak_src = gpu_arm(args, rank, world, local_rank, precisions)
    if rank != 0:
        return
    head = "mixed" if "mixed" in results else "fp64"
    res = results[head]
    ms = res["ms"]
    line = {
        "metric": METRIC, "value": res["value"], "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": statistics.mean(ms), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if head == "fp64" else "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "batch_per_gpu": args.batch, "lanes": res["tuning"]["lanes"],
                   "loop_on_device": res["tuning"]["loop_on_device"], "tuning": res["tuning"]["source"],
                   "selector": args.selector, "precision": head,
                   "refine_steps": args.refine_steps,
                   "l2": "flushed (256 MiB write) between timed steps", "parallelism": "replicas"},
        "latency_ms": {"p50": statistics.median(ms), "p99": sorted(ms)[min(len(ms) - 1, int(0.99 * len(ms)))],
                       "note": "per step; every solve of a batch completes at the end of its step"},
        "gpu_launches": res["launches"],
        "clocks": res["clocks"],
    }
    for prec, r in results.items():
        line[f"{prec}_solves_per_s"] = r["value"]
        line[f"{prec}_iterations_mean"] = statistics.mean(i["iterations"] for i in r["infos"])
        line[f"{prec}_rank_mean"] = statistics.mean(i["rank"] for i in r["infos"])
    if "mixed" in results and "fp64" in results:
        line["mixed_over_fp64"] = results["mixed"]["value"] / results["fp64"]["value"]
    if "e2e" in res:
        line["e2e"] = res["e2e"]
    line["roofline"] = roofline(res, head, hbm_peak, peak_src, args.batch)
    line["class_roofline"] = class_rooflines(res, head, hbm_peak)
    line["kernel_ms"] = {k: round(v[1], 3) for k, v in res["kernels"].items()}
    line["latency_bound_ms"] = {k: round(v[1], 3) for k, v in res["kernels"].items()
                                if k != "all" and v[2] + v[3] == 0 and v[1] > 0}
    if args.mixed_sizes > 0:
        line["mixed_sizes_batch"] = mixed_sizes_batch(args, rank)
        kept_multi, line["mixed_sizes_one_launch"] = mixed_sizes_one_launch(args, rank)
    kept = []
    if args.mixed_sizes <= 0:
        kept_multi = []
    if args.serve_requests > 0:
        line["serving"], kept = serving_stream(args, rank, lanes=args.serve_lanes)
    if not args.no_cpu and world == 1:
        cb, errs = cpu_baseline(rhss, replica_seeds(rank, args.batch), args.cpu_seconds, results,
                                args.err_check, pool)
        if kept:
            line["serving"]["accuracy"] = check_served(kept, pool)
        if kept_multi:
            line["mixed_sizes_one_launch"]["accuracy"] = check_served(
                kept_multi, pool, "every eighth problem of the batch with n <= 4095, exact sums")
        pool.close()
        line["cpu_baseline"] = cb
        line["rel_err_vs_exact"] = errs
        bad = {p: e["above_1e-6"] for p, e in errs.items() if e["above_1e-6"] > 0}
        line["accuracy"] = {"bar": ERR_BAR, "checked": {p: e["checked"] for p, e in errs.items()},
                            "passed": not bad}
        if bad:
            # a throughput at the metric's bar is not valid when a checked result misses the bar
            line["invalid"] = f"results above rel err {ERR_BAR:g}: {bad}"
    print(json.dumps(line))


if __name__ == "__main__":
    main()

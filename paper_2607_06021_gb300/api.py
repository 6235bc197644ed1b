"""PyTorch-tensor convenience layer over the C ABI (allocation and marshalling only)."""
from __future__ import annotations

import ctypes

import torch

from . import (INFO_BYTES, KERNEL_CLASSES, LRP_FP64, LRP_MIXED, LRP_NOT_CONVERGED, LRP_OK, LRP_SEL_BERNOULLI,
               LRP_SEL_LEVERAGE,
               LRP_SEL_QDEIM,
               LRP_RANK_CAPPED, lrp_default_opts, lrp_dst1, lrp_info, lrp_plan, lrp_plan_destroy,
               lrp_plan_kernel_stats, lrp_plan_kernel_work, lrp_plan_reset_stats, lrp_plan_set_timing,
               lrp_plan_set_trace, lrp_plan_trace, lrp_plan_pack, lrp_group_create, lrp_group_destroy,
               lrp_group_pack, lrp_group_plan, lrp_group_solve,
               lrp_plan_workspace_bytes, lrp_problem, lrp_solve_batch, lrp_warm_create,
               lrp_warm_destroy, lrp_warm_reset, lrp_poll, lrp_request, lrp_server_create,
               lrp_server_default_opts, lrp_server_destroy, lrp_server_get_stats, lrp_server_reset_stats,
               lrp_server_last_error, lrp_submit, lrp_wait, lrp_multi_create, lrp_multi_solve, lrp_multi_plan,
               lrp_multi_destroy)


def colmajor(x: torch.Tensor) -> torch.Tensor:
    """Column-major copy of a 2-D tensor (strides (1, rows))."""
    return x.t().contiguous().t()


def _ld(t: torch.Tensor) -> int:
    if t.dim() != 2 or t.dtype != torch.float64 or not t.is_cuda:
        raise ValueError("expected a 2-D CUDA float64 tensor")
    if t.shape[0] > 1 and t.stride(0) != 1:
        raise ValueError("expected a column-major tensor (stride(0) == 1)")
    return int(t.stride(1)) if t.shape[1] > 1 else int(t.shape[0])


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def parse_info(raw: torch.Tensor) -> dict:
    b = bytes(raw.cpu().numpy().tobytes())
    inf = lrp_info.from_buffer_copy(b)
    return {f: getattr(inf, f) for f, _ in lrp_info._fields_}


class Plan:
    """A solver plan for grids with n interior points per dimension."""

    def __init__(self, n: int, tol: float, max_rank: int, precision: str = "fp64", batch: int = 1,
                 max_rhs_rank: int = 64, max_iter: int = 30, m_cap: int = 0, seed: int = 0,
                 check_every: int = 1, refine_steps: int = 2, selector: str = "bernoulli", sample_factor: float = 1.0,
                 matrix: str = "poisson", loop_on_device: bool = False, gemm_rows_per_thread: int = 0,
                 dst_cta_threads: int = 0):
        o = lrp_default_opts()
        o.precision = LRP_FP64 if precision == "fp64" else LRP_MIXED
        o.batch = batch
        o.max_rhs_rank = max_rhs_rank
        o.max_iter = max_iter
        o.m_cap = m_cap
        o.seed = seed
        o.check_every = check_every
        o.refine_steps = refine_steps
        o.selector = {"ls": LRP_SEL_LEVERAGE, "qdeim": LRP_SEL_QDEIM, "bernoulli": LRP_SEL_BERNOULLI}[selector]
        o.sample_factor = sample_factor
        o.matrix = {"poisson": 0, "hilbert": 1, "k": 2}[matrix]
        o.loop_on_device = 1 if loop_on_device else 0
        o.gemm_rows_per_thread = gemm_rows_per_thread
        o.dst_cta_threads = dst_cta_threads
        self.n, self.tol, self.max_rank, self.batch = n, tol, max_rank, batch
        self.handle = lrp_plan(n, tol, max_rank, o)

    @property
    def workspace_bytes(self) -> int:
        return lrp_plan_workspace_bytes(self.handle)

    def set_timing(self, enable: bool) -> None:
        lrp_plan_set_timing(self.handle, enable)

    def pack(self, packed: torch.Tensor, offsets: torch.Tensor, stream=None) -> None:
        """Compact results of the last solve into packed (float64) and offsets (int64, count + 1)."""
        if packed.dtype != torch.float64 or offsets.dtype != torch.int64 or not packed.is_cuda or not offsets.is_cuda:
            raise ValueError("packed: CUDA float64, offsets: CUDA int64")
        lrp_plan_pack(self.handle, ctypes.c_void_p(packed.data_ptr()), packed.numel(),
                      ctypes.c_void_p(offsets.data_ptr()), _stream(stream))

    def set_trace(self, enable: bool) -> None:
        lrp_plan_set_trace(self.handle, enable)

    def trace(self, slot: int = 0):
        return lrp_plan_trace(self.handle, slot)

    def reset_stats(self) -> None:
        lrp_plan_reset_stats(self.handle)

    def kernel_stats(self) -> dict:
        """{class: (launches, total_ms, algorithmic_flops, algorithmic_bytes)} since the last reset."""
        out = {}
        for i, name in enumerate(KERNEL_CLASSES):
            out[name] = lrp_plan_kernel_stats(self.handle, i) + lrp_plan_kernel_work(self.handle, i)
        out["all"] = lrp_plan_kernel_stats(self.handle, -1) + lrp_plan_kernel_work(self.handle, -1)
        return out

    def close(self):
        if self.handle is not None:
            lrp_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def alloc_outputs(self, device="cuda"):
        n, r = self.n, self.max_rank
        U = torch.zeros((r, n), dtype=torch.float64, device=device).t()
        V = torch.zeros((r, n), dtype=torch.float64, device=device).t()
        S = torch.zeros(r, dtype=torch.float64, device=device)
        info = torch.zeros(INFO_BYTES, dtype=torch.uint8, device=device)
        return U, S, V, info

    def warm_record(self) -> "WarmRecord":
        return WarmRecord(self)

    def problem(self, U_f, s_f, V_f, outs, warm=None) -> lrp_problem:
        U, S, V, info = outs
        p = lrp_problem()
        p.warm = warm.handle if warm is not None else None
        p.r_f = int(U_f.shape[1])
        p.d_U_f, p.ldu_f = U_f.data_ptr(), _ld(U_f)
        p.d_s_f = s_f.data_ptr()
        p.d_V_f, p.ldv_f = V_f.data_ptr(), _ld(V_f)
        p.d_U, p.ldu = U.data_ptr(), _ld(U)
        p.d_S = S.data_ptr()
        p.d_V, p.ldv = V.data_ptr(), _ld(V)
        p.d_info = info.data_ptr()
        return p

    def solve_batch_into(self, inputs, outputs, stream=None, warms=None) -> None:
        """Enqueue a batch; inputs/outputs are lists of (U_f, s_f, V_f) / alloc_outputs()."""
        warms = warms if warms is not None else [None] * len(inputs)
        probs = [self.problem(*i, o, w) for i, o, w in zip(inputs, outputs, warms)]
        lrp_solve_batch(self.handle, probs, _stream(stream))

    def solve_batch(self, inputs, stream=None, warms=None):
        outs = [self.alloc_outputs() for _ in inputs]
        self.solve_batch_into(inputs, outs, stream, warms)
        torch.cuda.synchronize()
        res = []
        for U, S, V, info in outs:
            inf = parse_info(info)
            r = inf["rank"]
            res.append((U[:, :r], S[:r], V[:, :r], inf))
        return res

    def solve(self, U_f, s_f, V_f, stream=None, warm=None):
        return self.solve_batch([(U_f, s_f, V_f)], stream, [warm])[0]


class WarmRecord:
    """Warm-start record (index sets and iterate of a previous solve) for a plan."""

    def __init__(self, plan: Plan):
        self.plan = plan
        self.handle = lrp_warm_create(plan.handle)

    def reset(self) -> None:
        lrp_warm_reset(self.handle)

    def close(self) -> None:
        if self.handle is not None:
            lrp_warm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve(U_f, s_f, V_f, tol: float, max_rank: int, **kw):
    """One-off solve: W ~= U diag(S) V^T for T W + W T = h^2 U_f diag(s_f) V_f^T."""
    n = U_f.shape[0]
    p = Plan(n, tol, max_rank, max_rhs_rank=max(int(U_f.shape[1]), 1), **kw)
    try:
        return p.solve(U_f, s_f, V_f)
    finally:
        p.close()


def dst1(X: torch.Tensor, stream=None) -> torch.Tensor:
    """Orthonormal DST-I of the columns of a column-major float64 CUDA tensor."""
    n, c = X.shape
    Y = torch.empty((c, n), dtype=torch.float64, device=X.device).t()
    lrp_dst1(n, c, X.data_ptr(), _ld(X), Y.data_ptr(), _ld(Y) if c > 1 else n, _stream(stream))
    return Y


__all__ = ["Group", "Multi", "Plan", "Server", "WarmRecord", "solve", "dst1", "colmajor", "parse_info", "LRP_OK", "LRP_NOT_CONVERGED", "LRP_RANK_CAPPED"]


class Server:
    """Request server (host factors in, host factors out); see lrp_server_create."""

    def __init__(self, memory_cap_bytes: int | None = None, lanes: int = 2, max_batch: int = 64,
                 max_queue: int = 65536, warm_capacity: int = 64):
        o = lrp_server_default_opts()
        if memory_cap_bytes is not None:
            o.memory_cap_bytes = int(memory_cap_bytes)
        o.lanes, o.max_batch, o.max_queue, o.warm_capacity = lanes, max_batch, max_queue, warm_capacity
        self.handle = lrp_server_create(o)
        self._outputs = {}

    def submit(self, U_f, s_f, V_f, tol: float, max_rank: int, precision: str = "mixed", warm_key: int = 0):
        """Ticket, or None when the server is full.  U_f, V_f: n x r_f host arrays."""
        import numpy as np
        U_f = np.asfortranarray(U_f, dtype=np.float64)
        V_f = np.asfortranarray(V_f, dtype=np.float64)
        s_f = np.ascontiguousarray(s_f, dtype=np.float64)
        n, r_f = U_f.shape
        U = np.empty((n, max_rank), order="F")
        S = np.empty(max_rank)
        V = np.empty((n, max_rank), order="F")
        req = lrp_request()
        req.n, req.r_f, req.max_rank, req.tol = n, r_f, max_rank, float(tol)
        req.precision = LRP_FP64 if precision == "fp64" else LRP_MIXED
        req.warm_key = int(warm_key)
        req.U_f, req.s_f, req.V_f = U_f.ctypes.data, s_f.ctypes.data, V_f.ctypes.data
        req.U, req.S, req.V = U.ctypes.data, S.ctypes.data, V.ctypes.data
        t = lrp_submit(self.handle, req)
        if t is not None:
            self._outputs[t] = (U, S, V)
        return t

    def _take(self, t, r):
        U, S, V = self._outputs.pop(t)
        k = r.rank
        return U[:, :k], S[:k], V[:, :k], {f: getattr(r, f) for f, _ in r._fields_}

    def poll(self, ticket: int):
        r = lrp_poll(self.handle, ticket)
        return None if r is None else self._take(ticket, r)

    def wait(self, ticket: int, timeout_s: float = 60.0):
        r = lrp_wait(self.handle, ticket, int(timeout_s * 1e6))
        return None if r is None else self._take(ticket, r)

    def stats(self) -> dict:
        st = lrp_server_get_stats(self.handle)
        return {f: getattr(st, f) for f, _ in st._fields_}

    def reset_stats(self) -> None:
        lrp_server_reset_stats(self.handle)

    def last_error(self) -> str:
        return lrp_server_last_error(self.handle)

    def close(self) -> None:
        if self.handle is not None:
            lrp_server_destroy(self.handle)
            self.handle = None
            self._outputs.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _LanePlan(Plan):
    """A lane's plan inside a Group (statistics only; owned by the group)."""

    def __init__(self, handle, n, tol, max_rank, batch):
        self.handle, self.n, self.tol, self.max_rank, self.batch = handle, n, tol, max_rank, batch

    def close(self):
        self.handle = None


class Group:
    """lrp_group_*: one batch solved as `lanes` concurrent sub-batches."""

    def __init__(self, n: int, tol: float, max_rank: int, lanes: int, precision: str = "fp64", batch: int = 1,
                 max_rhs_rank: int = 64, max_iter: int = 30, m_cap: int = 0, seed: int = 0, selector: str = "bernoulli",
                 sample_factor: float = 1.0, matrix: str = "poisson", refine_steps: int = 2,
                 loop_on_device: bool = False, gemm_rows_per_thread: int = 0, dst_cta_threads: int = 0):
        o = lrp_default_opts()
        o.precision = LRP_FP64 if precision == "fp64" else LRP_MIXED
        o.refine_steps = refine_steps
        o.batch, o.max_rhs_rank, o.max_iter, o.m_cap, o.seed = batch, max_rhs_rank, max_iter, m_cap, seed
        o.selector = {"ls": LRP_SEL_LEVERAGE, "qdeim": LRP_SEL_QDEIM, "bernoulli": LRP_SEL_BERNOULLI}[selector]
        o.sample_factor = sample_factor
        o.matrix = {"poisson": 0, "hilbert": 1, "k": 2}[matrix]
        o.loop_on_device = 1 if loop_on_device else 0
        o.gemm_rows_per_thread = gemm_rows_per_thread
        o.dst_cta_threads = dst_cta_threads
        self.n, self.tol, self.max_rank, self.batch, self.lanes = n, tol, max_rank, batch, lanes
        self.handle = lrp_group_create(n, tol, max_rank, o, lanes)
        per = (batch + lanes - 1) // lanes
        self.plans = [_LanePlan(lrp_group_plan(self.handle, l), n, tol, max_rank, per) for l in range(lanes)]

    def alloc_outputs(self, device="cuda"):
        return self.plans[0].alloc_outputs(device)

    def solve_batch_into(self, inputs, outputs, stream=None) -> None:
        probs = [self.plans[0].problem(*i, o) for i, o in zip(inputs, outputs)]
        lrp_group_solve(self.handle, probs, _stream(stream))

    def solve_batch(self, inputs, stream=None):
        outs = [self.alloc_outputs() for _ in inputs]
        self.solve_batch_into(inputs, outs, stream)
        torch.cuda.synchronize()
        res = []
        for U, S, V, info in outs:
            inf = parse_info(info)
            r = inf["rank"]
            res.append((U[:, :r], S[:r], V[:, :r], inf))
        return res

    def pack(self, packed: torch.Tensor, offsets: torch.Tensor, stream=None) -> None:
        lrp_group_pack(self.handle, ctypes.c_void_p(packed.data_ptr()), packed.numel(),
                       ctypes.c_void_p(offsets.data_ptr()), _stream(stream))

    def kernel_stats(self) -> dict:
        """Launch counts summed over the lanes (and times / work, see Plan.kernel_stats)."""
        tot = None
        for p in self.plans:
            st = p.kernel_stats()
            tot = st if tot is None else {k: tuple(a + b for a, b in zip(tot[k], st[k])) for k in tot}
        return tot

    def reset_stats(self) -> None:
        for p in self.plans:
            p.reset_stats()

    def set_timing(self, enable: bool) -> None:
        for p in self.plans:
            p.set_timing(enable)

    def close(self) -> None:
        if self.handle is not None:
            for p in self.plans:
                p.close()
            lrp_group_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Multi:
    """lrp_multi_*: problems of several grid sizes solved as one CUDA graph launch."""

    def __init__(self, ns, batches, tol: float, max_rank: int, precision: str = "mixed", max_rhs_rank: int = 64,
                 max_iter: int = 30, m_cap: int = 0, seed: int = 0, selector: str = "bernoulli", sample_factor: float = 1.0,
                 refine_steps: int = 2):
        o = lrp_default_opts()
        o.precision = LRP_FP64 if precision == "fp64" else LRP_MIXED
        o.refine_steps = refine_steps
        o.max_rhs_rank, o.max_iter, o.m_cap, o.seed = max_rhs_rank, max_iter, m_cap, seed
        o.selector = {"ls": LRP_SEL_LEVERAGE, "qdeim": LRP_SEL_QDEIM, "bernoulli": LRP_SEL_BERNOULLI}[selector]
        o.sample_factor = sample_factor
        self.ns, self.tol, self.max_rank = list(ns), tol, max_rank
        self.handle = lrp_multi_create(self.ns, batches, tol, max_rank, o)
        self.plans = [_LanePlan(lrp_multi_plan(self.handle, i), n, tol, max_rank, b)
                      for i, (n, b) in enumerate(zip(self.ns, batches))]

    def alloc_outputs(self, n: int, device="cuda"):
        r = self.max_rank
        U = torch.zeros((r, n), dtype=torch.float64, device=device).t()
        V = torch.zeros((r, n), dtype=torch.float64, device=device).t()
        S = torch.zeros(r, dtype=torch.float64, device=device)
        info = torch.zeros(INFO_BYTES, dtype=torch.uint8, device=device)
        return U, S, V, info

    def solve_batch_into(self, inputs, outputs, stream=None) -> None:
        """inputs: list of (U_f, s_f, V_f) of any sizes in the set; outputs: alloc_outputs(n) each."""
        probs = [self.plans[0].problem(*i, o) for i, o in zip(inputs, outputs)]
        lrp_multi_solve(self.handle, [int(i[0].shape[0]) for i in inputs], probs, _stream(stream))

    def solve_batch(self, inputs, stream=None):
        outs = [self.alloc_outputs(int(i[0].shape[0])) for i in inputs]
        self.solve_batch_into(inputs, outs, stream)
        torch.cuda.synchronize()
        res = []
        for U, S, V, info in outs:
            inf = parse_info(info)
            r = inf["rank"]
            res.append((U[:, :r], S[:r], V[:, :r], inf))
        return res

    def kernel_stats(self) -> dict:
        tot = None
        for p in self.plans:
            st = p.kernel_stats()
            tot = st if tot is None else {k: tuple(a + b for a, b in zip(tot[k], st[k])) for k in tot}
        return tot

    def close(self) -> None:
        if self.handle is not None:
            for p in self.plans:
                p.close()
            lrp_multi_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

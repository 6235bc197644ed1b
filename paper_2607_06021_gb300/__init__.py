"""Python binding of liblrp.so (include/lrp.h): argument marshalling only.

Every computation runs in the library's sm_103a kernels.  PyTorch provides
device memory and streams.  Factor matrices are column-major: an n x r matrix
is a CUDA float64 tensor of shape (n, r) with strides (1, ld), ld >= n (for
example ``torch.empty(r, n).T``).  If the shared library is missing the import
of this package fails; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblrp.so")

LRP_OK, LRP_EINVAL, LRP_ENOMEM, LRP_ECUDA, LRP_ETIMEDOUT = 0, 1, 2, 3, 4
LRP_NOT_CONVERGED, LRP_RANK_CAPPED, LRP_EAGAIN, LRP_ECAPACITY = 5, 6, 7, 8
LRP_FP64, LRP_MIXED = 0, 1
LRP_SEL_LEVERAGE, LRP_SEL_QDEIM, LRP_SEL_BERNOULLI = 0, 1, 2
LRP_MAT_POISSON, LRP_MAT_HILBERT, LRP_MAT_K = 0, 1, 2
KERNEL_CLASSES = ["dst", "cross", "gram", "reduce", "gemm", "leverage", "chol", "core", "select", "stop",
                  "other", "refine", "gram_f32", "gemm_f32", "gram_df", "gemm_df", "dst_df"]


class LrpError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)}: {last_error()}")


class lrp_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("selector", ctypes.c_int32),
                ("max_iter", ctypes.c_int32), ("refine_steps", ctypes.c_int32),
                ("max_rhs_rank", ctypes.c_int32), ("batch", ctypes.c_int32),
                ("m_cap", ctypes.c_int32), ("check_every", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("sample_factor", ctypes.c_double),
                ("matrix", ctypes.c_int32), ("loop_on_device", ctypes.c_int32),
                ("gemm_rows_per_thread", ctypes.c_int32), ("dst_cta_threads", ctypes.c_int32)]


class lrp_info(ctypes.Structure):
    _fields_ = [("rank", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("status", ctypes.c_int32), ("r_star", ctypes.c_int32),
                ("size_I", ctypes.c_int32), ("size_J", ctypes.c_int32),
                ("total_iterations", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("rho", ctypes.c_double), ("eta_smin", ctypes.c_double),
                ("sigma_max", ctypes.c_double), ("reserved1", ctypes.c_double)]


class lrp_problem(ctypes.Structure):
    _fields_ = [("r_f", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("d_U_f", ctypes.c_void_p), ("ldu_f", ctypes.c_int64),
                ("d_s_f", ctypes.c_void_p), ("d_V_f", ctypes.c_void_p),
                ("ldv_f", ctypes.c_int64), ("d_U", ctypes.c_void_p), ("ldu", ctypes.c_int64),
                ("d_S", ctypes.c_void_p), ("d_V", ctypes.c_void_p), ("ldv", ctypes.c_int64),
                ("d_info", ctypes.c_void_p), ("warm", ctypes.c_void_p)]


class lrp_server_opts(ctypes.Structure):
    _fields_ = [("memory_cap_bytes", ctypes.c_int64), ("lanes", ctypes.c_int32),
                ("max_batch", ctypes.c_int32), ("max_queue", ctypes.c_int32),
                ("warm_capacity", ctypes.c_int32)]


class lrp_request(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("r_f", ctypes.c_int32), ("max_rank", ctypes.c_int32),
                ("tol", ctypes.c_double), ("precision", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("warm_key", ctypes.c_uint64), ("U_f", ctypes.c_void_p), ("s_f", ctypes.c_void_p),
                ("V_f", ctypes.c_void_p), ("U", ctypes.c_void_p), ("S", ctypes.c_void_p),
                ("V", ctypes.c_void_p)]


class lrp_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("rank", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("warm_used", ctypes.c_int32), ("latency_us", ctypes.c_double), ("queue_us", ctypes.c_double)]


class lrp_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("rejected", ctypes.c_int64),
                ("queued", ctypes.c_int64), ("running", ctypes.c_int64), ("plans", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("admitted_bytes", ctypes.c_int64),
                ("p50_us", ctypes.c_double), ("p99_us", ctypes.c_double), ("mean_us", ctypes.c_double),
                ("max_us", ctypes.c_double)]


INFO_BYTES = ctypes.sizeof(lrp_info)


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python paper_2607_06021_gb300/build.py` (no CPU fallback exists)")
    lib = ctypes.CDLL(LIB_PATH)
    P, I32, I64, D, VP = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
    sig = {
        "lrp_default_opts": ([ctypes.POINTER(lrp_opts)], I32),
        "lrp_plan": ([ctypes.POINTER(P), I64, D, I32, ctypes.POINTER(lrp_opts)], I32),
        "lrp_plan_destroy": ([P], I32),
        "lrp_warm_create": ([P, ctypes.POINTER(P)], I32),
        "lrp_warm_reset": ([P], I32),
        "lrp_warm_destroy": ([P], I32),
        "lrp_plan_workspace_bytes": ([P, ctypes.POINTER(ctypes.c_size_t)], I32),
        "lrp_solve": ([P, I32, VP, I64, VP, VP, I64, VP, I64, VP, VP, I64, VP, VP], I32),
        "lrp_solve_batch": ([P, I32, ctypes.POINTER(lrp_problem), VP], I32),
        "lrp_dst1": ([I64, I32, VP, I64, VP, I64, VP], I32),
        "lrp_dst1_noalloc": ([I64, I32, VP, I64, VP, I64, VP], I32),
        "lrp_plan_set_timing": ([P, I32], I32),
        "lrp_plan_set_trace": ([P, I32], I32),
        "lrp_plan_trace": ([P, I32, ctypes.POINTER(ctypes.c_double), I32, ctypes.POINTER(I32)], I32),
        "lrp_plan_kernel_stats": ([P, I32, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)], I32),
        "lrp_plan_reset_stats": ([P], I32),
        "lrp_plan_kernel_work": ([P, I32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)], I32),
        "lrp_plan_pack": ([P, VP, I64, VP, VP], I32),
        "lrp_group_create": ([ctypes.POINTER(P), I64, D, I32, ctypes.POINTER(lrp_opts), I32], I32),
        "lrp_group_solve": ([P, I32, ctypes.POINTER(lrp_problem), VP], I32),
        "lrp_group_plan": ([P, I32, ctypes.POINTER(P)], I32),
        "lrp_group_pack": ([P, VP, I64, VP, VP], I32),
        "lrp_group_destroy": ([P], I32),
        "lrp_multi_create": ([ctypes.POINTER(P), I32, ctypes.POINTER(I64), ctypes.POINTER(I32), D, I32,
                              ctypes.POINTER(lrp_opts)], I32),
        "lrp_multi_solve": ([P, I32, ctypes.POINTER(I64), ctypes.POINTER(lrp_problem), VP], I32),
        "lrp_multi_plan": ([P, I32, ctypes.POINTER(P)], I32),
        "lrp_multi_destroy": ([P], I32),
        "lrp_plan_estimate_bytes": ([I64, D, I32, ctypes.POINTER(lrp_opts), ctypes.POINTER(ctypes.c_size_t)], I32),
        "lrp_server_default_opts": ([ctypes.POINTER(lrp_server_opts)], I32),
        "lrp_request_footprint": ([I64, I32, I32], ctypes.c_size_t),
        "lrp_server_create": ([ctypes.POINTER(P), ctypes.POINTER(lrp_server_opts)], I32),
        "lrp_submit": ([P, ctypes.POINTER(lrp_request), ctypes.POINTER(ctypes.c_uint64)], I32),
        "lrp_poll": ([P, ctypes.c_uint64, ctypes.POINTER(lrp_result)], I32),
        "lrp_wait": ([P, ctypes.c_uint64, ctypes.POINTER(lrp_result), I64], I32),
        "lrp_server_get_stats": ([P, ctypes.POINTER(lrp_server_stats)], I32),
        "lrp_server_reset_stats": ([P], I32),
        "lrp_server_last_error": ([P, ctypes.c_char_p, ctypes.c_size_t], I32),
        "lrp_server_destroy": ([P], I32),
        "lrp_last_error": ([], ctypes.c_char_p),
        "lrp_status_string": ([I32], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


_lib = _load()


def library():
    return _lib


def last_error() -> str:
    return _lib.lrp_last_error().decode()


def status_string(s: int) -> str:
    return _lib.lrp_status_string(int(s)).decode()


def _check(s: int, where: str, ok=(LRP_OK,)):
    if s not in ok:
        raise LrpError(s, where)
    return s


def lrp_default_opts() -> lrp_opts:
    o = lrp_opts()
    _check(_lib.lrp_default_opts(ctypes.byref(o)), "lrp_default_opts")
    return o


def lrp_plan(n: int, tol: float, max_rank: int, opts: lrp_opts | None = None):
    h = ctypes.c_void_p()
    _check(_lib.lrp_plan(ctypes.byref(h), int(n), float(tol), int(max_rank),
                         ctypes.byref(opts) if opts is not None else None), "lrp_plan")
    return h


def lrp_group_create(n: int, tol: float, max_rank: int, opts: lrp_opts, lanes: int):
    h = ctypes.c_void_p()
    _check(_lib.lrp_group_create(ctypes.byref(h), int(n), float(tol), int(max_rank), ctypes.byref(opts), int(lanes)),
           "lrp_group_create")
    return h


def lrp_group_solve(group, problems, stream) -> int:
    arr = (lrp_problem * len(problems))(*problems)
    return _check(_lib.lrp_group_solve(group, len(problems), arr, stream), "lrp_group_solve")


def lrp_group_plan(group, lane: int):
    h = ctypes.c_void_p()
    _check(_lib.lrp_group_plan(group, int(lane), ctypes.byref(h)), "lrp_group_plan")
    return h


def lrp_group_pack(group, d_packed, capacity: int, d_offsets, stream) -> None:
    _check(_lib.lrp_group_pack(group, d_packed, int(capacity), d_offsets, stream), "lrp_group_pack")


def lrp_group_destroy(group) -> None:
    _check(_lib.lrp_group_destroy(group), "lrp_group_destroy")


def lrp_multi_create(ns, batches, tol: float, max_rank: int, opts: lrp_opts):
    h = ctypes.c_void_p()
    a = (ctypes.c_int64 * len(ns))(*[int(v) for v in ns])
    b = (ctypes.c_int32 * len(batches))(*[int(v) for v in batches])
    _check(_lib.lrp_multi_create(ctypes.byref(h), len(ns), a, b, float(tol), int(max_rank), ctypes.byref(opts)),
           "lrp_multi_create")
    return h


def lrp_multi_solve(multi, ns, problems, stream) -> int:
    a = (ctypes.c_int64 * len(ns))(*[int(v) for v in ns])
    arr = (lrp_problem * len(problems))(*problems)
    return _check(_lib.lrp_multi_solve(multi, len(problems), a, arr, stream), "lrp_multi_solve")


def lrp_multi_plan(multi, index: int):
    h = ctypes.c_void_p()
    _check(_lib.lrp_multi_plan(multi, int(index), ctypes.byref(h)), "lrp_multi_plan")
    return h


def lrp_multi_destroy(multi) -> None:
    _check(_lib.lrp_multi_destroy(multi), "lrp_multi_destroy")


def lrp_plan_pack(plan, d_packed, capacity: int, d_offsets, stream) -> None:
    _check(_lib.lrp_plan_pack(plan, d_packed, int(capacity), d_offsets, stream), "lrp_plan_pack")


def lrp_plan_estimate_bytes(n: int, tol: float, max_rank: int, opts: lrp_opts | None = None) -> int:
    v = ctypes.c_size_t()
    _check(_lib.lrp_plan_estimate_bytes(int(n), float(tol), int(max_rank),
                                        ctypes.byref(opts) if opts is not None else None, ctypes.byref(v)),
           "lrp_plan_estimate_bytes")
    return int(v.value)


def lrp_server_default_opts() -> lrp_server_opts:
    o = lrp_server_opts()
    _check(_lib.lrp_server_default_opts(ctypes.byref(o)), "lrp_server_default_opts")
    return o


def lrp_request_footprint(n: int, r_f: int, max_rank: int) -> int:
    return int(_lib.lrp_request_footprint(int(n), int(r_f), int(max_rank)))


def lrp_server_create(opts: lrp_server_opts | None = None):
    h = ctypes.c_void_p()
    _check(_lib.lrp_server_create(ctypes.byref(h), ctypes.byref(opts) if opts is not None else None),
           "lrp_server_create")
    return h


def lrp_submit(server, req: lrp_request):
    """Ticket, or None when the server answers LRP_EAGAIN (full: retry later)."""
    t = ctypes.c_uint64()
    s = _check(_lib.lrp_submit(server, ctypes.byref(req), ctypes.byref(t)), "lrp_submit", (LRP_OK, LRP_EAGAIN))
    return int(t.value) if s == LRP_OK else None


def lrp_poll(server, ticket: int):
    """lrp_result once finished, else None."""
    r = lrp_result()
    s = _check(_lib.lrp_poll(server, ctypes.c_uint64(ticket), ctypes.byref(r)), "lrp_poll", (LRP_OK, LRP_EAGAIN))
    return r if s == LRP_OK else None


def lrp_wait(server, ticket: int, timeout_us: int):
    r = lrp_result()
    s = _check(_lib.lrp_wait(server, ctypes.c_uint64(ticket), ctypes.byref(r), int(timeout_us)), "lrp_wait",
               (LRP_OK, LRP_ETIMEDOUT))
    return r if s == LRP_OK else None


def lrp_server_get_stats(server) -> lrp_server_stats:
    st = lrp_server_stats()
    _check(_lib.lrp_server_get_stats(server, ctypes.byref(st)), "lrp_server_get_stats")
    return st


def lrp_server_last_error(server) -> str:
    buf = ctypes.create_string_buffer(1024)
    _check(_lib.lrp_server_last_error(server, buf, 1024), "lrp_server_last_error")
    return buf.value.decode()


def lrp_server_reset_stats(server) -> None:
    _check(_lib.lrp_server_reset_stats(server), "lrp_server_reset_stats")


def lrp_server_destroy(server) -> None:
    _check(_lib.lrp_server_destroy(server), "lrp_server_destroy")


def lrp_warm_create(plan):
    h = ctypes.c_void_p()
    _check(_lib.lrp_warm_create(plan, ctypes.byref(h)), "lrp_warm_create")
    return h


def lrp_warm_reset(warm) -> None:
    _check(_lib.lrp_warm_reset(warm), "lrp_warm_reset")


def lrp_warm_destroy(warm) -> None:
    _check(_lib.lrp_warm_destroy(warm), "lrp_warm_destroy")


def lrp_plan_destroy(plan) -> None:
    _check(_lib.lrp_plan_destroy(plan), "lrp_plan_destroy")


def lrp_plan_workspace_bytes(plan) -> int:
    v = ctypes.c_size_t()
    _check(_lib.lrp_plan_workspace_bytes(plan, ctypes.byref(v)), "lrp_plan_workspace_bytes")
    return int(v.value)


def lrp_solve(plan, r_f, d_U_f, ldu_f, d_s_f, d_V_f, ldv_f, d_U, ldu, d_S, d_V, ldv, d_info, stream) -> int:
    return _check(_lib.lrp_solve(plan, int(r_f), d_U_f, int(ldu_f), d_s_f, d_V_f, int(ldv_f), d_U, int(ldu),
                                 d_S, d_V, int(ldv), d_info, stream), "lrp_solve")


def lrp_solve_batch(plan, problems, stream) -> int:
    arr = (lrp_problem * len(problems))(*problems)
    return _check(_lib.lrp_solve_batch(plan, len(problems), arr, stream), "lrp_solve_batch")


def lrp_dst1(n, ncols, d_X, ldx, d_Y, ldy, stream) -> int:
    return _check(_lib.lrp_dst1(int(n), int(ncols), d_X, int(ldx), d_Y, int(ldy), stream), "lrp_dst1")


def lrp_dst1_noalloc(n, ncols, d_X, ldx, d_Y, ldy, stream) -> int:
    """lrp_dst1 for callers that cannot allocate device memory (n+1 <= 8192)."""
    return _check(_lib.lrp_dst1_noalloc(int(n), int(ncols), d_X, int(ldx), d_Y, int(ldy), stream),
                  "lrp_dst1_noalloc")


def lrp_plan_set_timing(plan, enable: bool) -> None:
    _check(_lib.lrp_plan_set_timing(plan, 1 if enable else 0), "lrp_plan_set_timing")


LRP_TRACE_LEN = 96
LRP_TRACE_WIDTH = 8
TRACE_FIELDS = ("iteration", "rho", "eta_smin", "size_I", "size_J", "rank", "snorm", "size_I_kept")


def lrp_plan_set_trace(plan, enable: bool) -> None:
    _check(_lib.lrp_plan_set_trace(plan, 1 if enable else 0), "lrp_plan_set_trace")


def lrp_plan_trace(plan, slot: int):
    """Rows of the slot's per-iteration trace, as dicts keyed by TRACE_FIELDS."""
    buf = (ctypes.c_double * (LRP_TRACE_LEN * LRP_TRACE_WIDTH))()
    cnt = ctypes.c_int32()
    _check(_lib.lrp_plan_trace(plan, slot, buf, LRP_TRACE_LEN, ctypes.byref(cnt)), "lrp_plan_trace")
    rows = []
    for i in range(cnt.value):
        row = buf[i * LRP_TRACE_WIDTH:(i + 1) * LRP_TRACE_WIDTH]
        rows.append({k: (int(v) if k not in ("rho", "eta_smin", "snorm") else float(v))
                     for k, v in zip(TRACE_FIELDS, row)})
    return rows


def lrp_plan_kernel_stats(plan, kclass: int):
    n = ctypes.c_int64()
    ms = ctypes.c_double()
    _check(_lib.lrp_plan_kernel_stats(plan, int(kclass), ctypes.byref(n), ctypes.byref(ms)),
           "lrp_plan_kernel_stats")
    return int(n.value), float(ms.value)


def lrp_plan_kernel_work(plan, kclass: int):
    f = ctypes.c_double()
    b = ctypes.c_double()
    _check(_lib.lrp_plan_kernel_work(plan, int(kclass), ctypes.byref(f), ctypes.byref(b)), "lrp_plan_kernel_work")
    return float(f.value), float(b.value)


def lrp_plan_reset_stats(plan) -> None:
    _check(_lib.lrp_plan_reset_stats(plan), "lrp_plan_reset_stats")


from .api import Group, Multi, Plan, Server, WarmRecord, dst1, colmajor, parse_info, solve  # noqa: E402,F401

"""The C-ABI library loads and exports every entry point that include/lrp.h declares
(no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lrp.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    names = re.findall(r"^\s*(?:lrp_status|const\s+char\s*\*)\s*(lrp_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = declared_functions()
    for required in ["lrp_plan", "lrp_solve", "lrp_solve_batch", "lrp_plan_destroy", "lrp_dst1",
                     "lrp_last_error", "lrp_default_opts"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    pkg = pytest.importorskip("paper_2607_06021_gb300")
    lib = ctypes.CDLL(pkg.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_side_argument_checks_need_no_gpu():
    pkg = pytest.importorskip("paper_2607_06021_gb300")
    o = pkg.lrp_default_opts()
    assert o.max_iter == 30 and o.precision == pkg.LRP_FP64
    lib = pkg.library()
    h = ctypes.c_void_p()
    # n+1 not a power of two, tol out of range, NULL out: rejected before any device call
    assert lib.lrp_plan(ctypes.byref(h), 100, 1e-8, 8, None) == pkg.LRP_EINVAL
    assert "power of two" in pkg.last_error()
    assert lib.lrp_plan(ctypes.byref(h), 255, 0.0, 8, None) == pkg.LRP_EINVAL
    assert lib.lrp_plan(None, 255, 1e-8, 8, None) == pkg.LRP_EINVAL
    assert lib.lrp_dst1(100, 1, None, 100, None, 100, None) == pkg.LRP_EINVAL
    assert pkg.status_string(pkg.LRP_RANK_CAPPED) == "LRP_RANK_CAPPED"


def test_option_checks_need_no_gpu():
    # Option combinations the library refuses on the host, before any device call.
    pkg = pytest.importorskip("paper_2607_06021_gb300")
    lib = pkg.library()
    h = ctypes.c_void_p()

    def plan(n=255, **kw):
        o = pkg.lrp_default_opts()
        for k, v in kw.items():
            setattr(o, k, v)
        return lib.lrp_plan(ctypes.byref(h), n, 1e-8, 8, ctypes.byref(o))

    assert pkg.lrp_default_opts().refine_steps == 2 and pkg.lrp_default_opts().sample_factor == 1.0
    assert pkg.lrp_default_opts().matrix == pkg.LRP_MAT_POISSON
    assert pkg.lrp_default_opts().selector == pkg.LRP_SEL_BERNOULLI
    assert pkg.lrp_default_opts().loop_on_device == 0
    assert plan(loop_on_device=2) == pkg.LRP_EINVAL and "loop_on_device" in pkg.last_error()
    assert plan(selector=7) == pkg.LRP_EINVAL and "selector" in pkg.last_error()
    assert plan(selector=pkg.LRP_SEL_BERNOULLI, sample_factor=0.0) == pkg.LRP_EINVAL
    assert plan(selector=pkg.LRP_SEL_BERNOULLI, sample_factor=-1.0) == pkg.LRP_EINVAL
    assert plan(matrix=9) == pkg.LRP_EINVAL and "matrix" in pkg.last_error()
    # the test matrices: FP64 only, any n (no transform), K needs two grid points
    assert plan(matrix=pkg.LRP_MAT_HILBERT, precision=pkg.LRP_MIXED) == pkg.LRP_EINVAL
    assert "FP64" in pkg.last_error()
    assert plan(n=1, matrix=pkg.LRP_MAT_K) == pkg.LRP_EINVAL
    assert plan(precision=pkg.LRP_MIXED, refine_steps=3, m_cap=64) == pkg.LRP_EINVAL
    assert "refine_steps" in pkg.last_error()
    # n + 1 need not be a power of two for a matrix given by entries: the host
    # checks pass and only the device step can fail here (no GPU)
    assert plan(n=300, matrix=pkg.LRP_MAT_HILBERT) in (pkg.LRP_OK, pkg.LRP_ECUDA)
    if h.value:
        lib.lrp_plan_destroy(h)


def test_struct_layouts_match_header():
    pkg = pytest.importorskip("paper_2607_06021_gb300")
    assert ctypes.sizeof(pkg.lrp_opts) == 64
    assert ctypes.sizeof(pkg.lrp_info) == 64
    assert ctypes.sizeof(pkg.lrp_problem) == 104
    assert ctypes.sizeof(pkg.lrp_server_opts) == 24
    assert ctypes.sizeof(pkg.lrp_request) == 88
    assert ctypes.sizeof(pkg.lrp_result) == 32
    assert ctypes.sizeof(pkg.lrp_server_stats) == 96


def test_plan_estimate_is_host_only_and_linear_in_batch():
    # Sizing runs without a device: the arena grows by the same amount per
    # batch slot, and mixed precision adds an FP32 workspace.
    pkg = pytest.importorskip("paper_2607_06021_gb300")
    o = pkg.lrp_default_opts()
    o.max_rhs_rank, o.m_cap = 20, 64
    sizes = []
    for b in (1, 2, 3, 8):
        o.batch = b
        sizes.append(pkg.lrp_plan_estimate_bytes(4095, 1e-8, 64, o))
    per = sizes[1] - sizes[0]
    # linear up to the 256-byte alignment of each of the arena's allocations
    assert per > 0 and abs((sizes[2] - sizes[1]) - per) <= 64 * 256
    assert abs((sizes[3] - sizes[0]) - 7 * per) <= 64 * 256
    # the five n x m_cap FP64 blocks per side dominate one slot
    assert per >= 2 * 5 * 4096 * 64 * 8
    o.batch, o.precision = 1, pkg.LRP_MIXED
    assert pkg.lrp_plan_estimate_bytes(4095, 1e-8, 64, o) > sizes[0]
    with pytest.raises(pkg.LrpError):
        pkg.lrp_plan_estimate_bytes(4000, 1e-8, 64, o)
    # a matrix given by entries: any n, and no transform scratch
    o.precision = pkg.LRP_FP64
    poisson_16k = pkg.lrp_plan_estimate_bytes(16383, 1e-8, 64, o)  # multi-pass transform: scratch
    o.matrix = pkg.LRP_MAT_HILBERT
    assert pkg.lrp_plan_estimate_bytes(4000, 1e-8, 64, o) > 0
    assert pkg.lrp_plan_estimate_bytes(4095, 1e-8, 64, o) == sizes[0]  # shared-memory transform: none
    assert pkg.lrp_plan_estimate_bytes(16383, 1e-8, 64, o) < poisson_16k


def test_request_footprint_formula():
    pkg = pytest.importorskip("paper_2607_06021_gb300")
    # 8 n (2 r_f + 4 m_cap + 2 max_rank), m_cap = min(2 max_rank + r_f rounded up to 16, 256)
    assert pkg.lrp_request_footprint(4095, 20, 64) == 8 * 4095 * (40 + 4 * 160 + 128)
    assert pkg.lrp_request_footprint(262143, 48, 128) == 8 * 262143 * (96 + 4 * 256 + 256)
    assert pkg.lrp_request_footprint(1023, 2, 8) == 8 * 1023 * (4 + 4 * 32 + 16)
    assert pkg.lrp_request_footprint(255, 0, 8) == 0


def test_launch_shape_options_are_checked():
    import paper_2607_06021_gb300 as pkg
    for field, bad in (("gemm_rows_per_thread", 3), ("gemm_rows_per_thread", -1), ("dst_cta_threads", 300),
                       ("dst_cta_threads", 2048)):
        o = pkg.lrp_default_opts()
        setattr(o, field, bad)
        with pytest.raises(pkg.LrpError):
            pkg.lrp_plan_estimate_bytes(4095, 1e-8, 64, o)
    o = pkg.lrp_default_opts()
    assert o.gemm_rows_per_thread == 0 and o.dst_cta_threads == 0
    o.gemm_rows_per_thread, o.dst_cta_threads = 1, 1024
    assert pkg.lrp_plan_estimate_bytes(4095, 1e-8, 64, o) == pkg.lrp_plan_estimate_bytes(4095, 1e-8, 64, None)

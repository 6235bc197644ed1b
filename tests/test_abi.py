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


def test_struct_layouts_match_header():
    pkg = pytest.importorskip("paper_2607_06021_gb300")
    assert ctypes.sizeof(pkg.lrp_opts) == 40
    assert ctypes.sizeof(pkg.lrp_info) == 64
    assert ctypes.sizeof(pkg.lrp_problem) == 104

"""The bench's roofline arithmetic (CPU): the derived ALU peaks follow from the
unit counts and from the rounding steps the double-float kernels actually
execute (counted in their sources), each class is held to the larger of its ALU
and HBM times, and the reported dominant class, fraction and traffic follow from
the kernel statistics."""
import math
import os
import re
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2607_06021_gb300", "csrc")
sys.path.insert(0, ROOT)

import bench  # noqa: E402

ROUNDED = re.compile(r"__(fadd|fsub|fmul|fmaf)_rn\(")


def _body(path: str, signature: str) -> str:
    """Source of the function whose definition starts with `signature`."""
    src = open(os.path.join(CSRC, path)).read()
    i = src.index(signature)
    j = src.index("{", i)
    depth = 0
    for k in range(j, len(src)):
        depth += {"{": 1, "}": -1}.get(src[k], 0)
        if depth == 0:
            return src[j:k + 1]
    raise AssertionError(signature)


def _steps(path: str, signature: str, two_sum_steps: int = 3) -> int:
    """FP32 instructions of a double-float routine: its rounded intrinsics, plus
    those of each fast TwoSum it calls."""
    body = _body(path, signature)
    return len(ROUNDED.findall(body)) + two_sum_steps * body.count("df_fast_two_sum(")


def test_fast_two_sum_is_three_steps():
    assert _steps("dfloat.cuh", "__device__ __forceinline__ dfloat df_fast_two_sum", 0) == 3


def test_double_float_instruction_counts_match_the_sources():
    add = _steps("dfloat.cuh", "__device__ __forceinline__ dfloat operator+(const dfloat& a, const dfloat& b)")
    mul = _steps("dfloat.cuh", "__device__ __forceinline__ dfloat operator*(const dfloat& a, const dfloat& b)")
    assert (add, mul) == (20, 7)
    # multiply-add of FP32 data into a (hi, lo) sum (the FP32 iterations' first Gram)
    assert _steps("tall.cu", "__device__ __forceinline__ void df_add_product") == 10
    # multiply-add of (hi, lo) data (the refinement's products and Grams)
    assert _steps("dfmat.cu", "__device__ __forceinline__ void dd_madd") == 13
    # radix-2 butterfly: a complex product (4 multiplies, 2 adds) and 4 adds, 10 flops
    assert (4 * mul + 6 * add) / 10 == pytest.approx(14.8)


def test_derived_peaks():
    lanes = 152 * 128 * 2.070 / 1e3  # FP32 lane instructions, 10^12 per second
    assert bench.FP64_PEAK_TFLOPS == pytest.approx(152 * 4 * 2.070 / 1e3)
    assert bench.FP64_PEAK_TFLOPS == pytest.approx(1.259, rel=1e-3)
    assert bench.FP32_PEAK_TFLOPS == pytest.approx(2 * lanes)
    assert bench.DF_MADD32_TFLOPS == pytest.approx(lanes / 10 * 2)
    assert bench.DF_MADD_TFLOPS == pytest.approx(lanes / 13 * 2)
    assert bench.DF_FFT_TFLOPS == pytest.approx(lanes / 14.8)
    assert set(bench.PIPES["mixed"].values()) <= set(bench.ALU_PEAKS)
    assert set(bench.PIPES["fp64"].values()) <= set(bench.ALU_PEAKS)


def test_class_bound_takes_the_larger_term():
    hbm = 6672.5
    # 1 GB in 1 ms on an FP32 class with little arithmetic: HBM-bound
    b = bench.class_bound("mixed", "gemm_f32", 10, 1.0, 1e9, 1e9, hbm)
    assert b["bound"] == "hbm" and b["unit"] == "GB/s"
    assert b["achieved"] == pytest.approx(1e9 / 1e-3 / 1e9)
    assert b["frac"] == pytest.approx(b["achieved"] / hbm)
    assert b["algorithmic_per_launch"] == pytest.approx(1e8)
    # the same bytes with 1 PFLOP of double-float work: ALU-bound on its own pipe
    b = bench.class_bound("mixed", "gram_df", 4, 500.0, 1e15, 1e9, hbm)
    assert b["bound"] == "alu" and b["pipe"] == "df32" and b["unit"] == "TFLOP/s"
    assert b["achieved"] == pytest.approx(1e15 / 0.5 / 1e12)
    assert b["frac"] == pytest.approx(b["achieved"] / bench.DF_MADD32_TFLOPS)
    # a class without an arithmetic pipe is held to HBM alone
    b = bench.class_bound("mixed", "refine", 1, 2.0, 1e15, 1e6, hbm)
    assert b["bound"] == "hbm"


def test_roofline_reports_the_dominant_class_and_scaled_traffic():
    hbm = 6672.5
    res = {"kernels": {"all": (100, 50.0, 0.0, 0.0),
                       "core": (10, 30.0, 0.0, 0.0),          # most time, but no algorithmic work
                       "gram_df": (8, 12.0, 8e12, 1e9),
                       "gemm_f32": (20, 10.0, 1e11, 4e10)}}
    r = bench.roofline(res, "mixed", hbm, "measured", 1024)
    assert r["kernel"] == "gram_df" and r["launches"] == 8
    assert r["avg_launch_us"] == pytest.approx(1500.0)
    assert r["traffic"] == pytest.approx(bench.TRAFFIC_B128[("mixed", "gram_df")][0] * 8)
    assert r["peak_source"] == bench.PEAK_SOURCE["df32"]
    cr = bench.class_rooflines(res, "mixed", hbm)
    assert set(cr) == {"gram_df", "gemm_f32"}
    assert cr["gram_df"]["bound"] == "alu_df32"
    assert cr["gemm_f32"]["bound"] == "hbm"
    assert math.isclose(cr["gemm_f32"]["frac"], round(4e10 / 0.01 / 1e9 / hbm, 4))

"""The integer-pipe FP64 <-> FP32 conversions of csrc/f64cvt.cuh, compiled as
plain C++ on the host and compared bit for bit with the C casts (IEEE 754
round to nearest, ties to even; the widening is exact).

The kernels use these routines in place of the hardware conversions (which
GB300 executes on its FP64 pipe), so they must give the same bits for every
input class: normal results, results that round into or out of the FP32
subnormal range, overflow to infinity, signed zeros, ties in both directions.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2607_06021_gb300", "csrc")

HARNESS = r"""
#include "f64cvt.cuh"
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>

static long bad = 0, checked = 0;

static void narrow(double x) {
  const float a = lrp::f64_to_f32_rn(x), b = (float)x;
  uint32_t ua, ub;
  memcpy(&ua, &a, 4);
  memcpy(&ub, &b, 4);
  ++checked;
  if (ua != ub && !(std::isnan(a) && std::isnan(b))) {
    if (bad < 5) printf("narrow %a: %08x vs %08x\n", x, ua, ub);
    ++bad;
  }
}

static void widen(float f) {
  const double a = lrp::f32_to_f64(f), b = (double)f;
  uint64_t ua, ub;
  memcpy(&ua, &a, 8);
  memcpy(&ub, &b, 8);
  ++checked;
  if (ua != ub && !(std::isnan(a) && std::isnan(b))) {
    if (bad < 5) printf("widen %a\n", (double)f);
    ++bad;
  }
}

int main() {
  std::mt19937_64 g(12345);
  // uniformly random bit patterns (every exponent class, NaNs included)
  for (int i = 0; i < 2000000; ++i) {
    const uint64_t b = g();
    double x;
    memcpy(&x, &b, 8);
    narrow(x);
  }
  // every FP64 exponent around the FP32 range, with the fraction patterns that
  // decide the rounding (exact ties, just above and below, all ones)
  const uint64_t pats[] = {0ull, 1ull << 28, (1ull << 28) - 1, (1ull << 28) + 1, 1ull << 29, (1ull << 29) | (1ull << 28),
                           0xfffffffffffffull, 0xfffffe0000000ull, 0xfffffefffffffull, 0xffffff0000000ull};
  for (uint64_t e = 850; e < 1200; ++e) {
    for (uint64_t s = 0; s < 2; ++s) {
      for (uint64_t p : pats) {
        double x;
        const uint64_t b = (s << 63) | (e << 52) | p;
        memcpy(&x, &b, 8);
        narrow(x);
      }
      for (int i = 0; i < 2000; ++i) {
        double x;
        const uint64_t b = (s << 63) | (e << 52) | (g() & 0xfffffffffffffull);
        memcpy(&x, &b, 8);
        narrow(x);
      }
    }
  }
  const double special[] = {0.0, -0.0, INFINITY, -INFINITY, 1e-300, -1e-300, 3.4028234663852886e38,
                            3.4028235677973366e38, 1.1754943508222875e-38, 1.401298464324817e-45,
                            7.006492321624085e-46, 7.006492321624087e-46};
  for (double x : special) narrow(x);
  // every FP32 bit pattern with the low 8 bits fixed, plus all subnormals
  for (uint64_t u = 0; u < (1ull << 32); u += 251) {
    const uint32_t b = (uint32_t)u;
    float f;
    memcpy(&f, &b, 4);
    widen(f);
  }
  for (uint32_t u = 0; u < (1u << 23); ++u) {
    for (uint32_t s = 0; s < 2; ++s) {
      const uint32_t b = (s << 31) | u;
      float f;
      memcpy(&f, &b, 4);
      widen(f);
    }
  }
  printf("checked %ld mismatches %ld\n", checked, bad);
  return bad != 0;
}
"""


def test_integer_conversions_match_the_c_casts(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "cvt.cpp"
    src.write_text(HARNESS)
    exe = tmp_path / "cvt"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    res = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stdout + res.stderr
    assert "mismatches 0" in res.stdout

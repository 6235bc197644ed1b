// Double-float numbers: an unevaluated sum hi + lo of two FP32 values (|lo| <=
// ulp(hi) / 2), about 48 significant bits, computed on the FP32 pipe.  GB300's
// FP32 pipe runs at 64x its FP64 pipe, so double-float arithmetic (a few FP32
// operations per operation) is several times faster than FP64 where ~1e-13
// relative accuracy suffices.
//
// Sums use Knuth's TwoSum and products the FMA-exact product (Dekker's
// algorithms in FMA form); the _rn intrinsics keep the compiler from
// contracting or reordering the error-free steps.
#pragma once
#include <cuda_runtime.h>

#include "f64cvt.cuh"

namespace lrp {

struct dfloat {
  float hi, lo;
  dfloat() = default;
  __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
  // The conversions to and from FP64 round exactly as the hardware ones but run
  // on the integer pipe (f64cvt.cuh); only the FP64 add/subtract remain.
  __device__ explicit dfloat(double x) {
    hi = f64_to_f32_rn(x);
    lo = f64_to_f32_rn(x - f32_to_f64(hi));
  }
  __device__ explicit dfloat(float x) : hi(x), lo(0.f) {}
  __device__ explicit dfloat(int x) : hi((float)x), lo(0.f) {}
  __device__ explicit operator double() const { return f32_to_f64(hi) + f32_to_f64(lo); }
  __device__ explicit operator float() const { return __fadd_rn(hi, lo); }
};

__device__ __forceinline__ dfloat df_fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return dfloat(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ dfloat operator+(const dfloat& a, const dfloat& b) {
  // TwoSum of the high parts and of the low parts, then two renormalisations
  float s = __fadd_rn(a.hi, b.hi);
  float bb = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  float t = __fadd_rn(a.lo, b.lo);
  float cc = __fsub_rn(t, a.lo);
  float f = __fadd_rn(__fsub_rn(a.lo, __fsub_rn(t, cc)), __fsub_rn(b.lo, cc));
  e = __fadd_rn(e, t);
  dfloat r = df_fast_two_sum(s, e);
  r.lo = __fadd_rn(r.lo, f);
  return df_fast_two_sum(r.hi, r.lo);
}

__device__ __forceinline__ dfloat operator-(const dfloat& a) { return dfloat(-a.hi, -a.lo); }
__device__ __forceinline__ dfloat operator-(const dfloat& a, const dfloat& b) { return a + (-b); }

__device__ __forceinline__ dfloat operator*(const dfloat& a, const dfloat& b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}

}  // namespace lrp

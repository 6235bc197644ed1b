// FP64 -> FP32 conversion with round-to-nearest-even on the integer pipe.
//
// GB300 executes the hardware FP64 -> FP32 conversion on its FP64 pipe, which
// retires 2 lanes per clock per SM (1/64 of the FP32 pipe).  Kernels that read
// FP64 data and compute in FP32 (the FP32 DST of the FP64 right-hand-side
// factors) would spend most of that pipe on conversions.  This routine gives
// the same IEEE 754 result (the nearest FP32 value, ties to even; overflow to
// infinity; results below the normal range rounded to FP32 subnormals) from
// the bit pattern with 32-bit integer operations; only infinities and NaNs
// take the hardware conversion.  Bit equality with the C cast `(float)x` is
// tested on the host over every exponent class (the routine compiles as plain
// C++ when this header is included without nvcc).
//
// IEEE 754 binary64: sign (1), biased exponent e (11, bias 1023), fraction (52).
// binary32: sign (1), biased exponent (8, bias 127), fraction (23).
#pragma once
#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define LRP_CVT_FN __host__ __device__ __forceinline__
#else
#define LRP_CVT_FN inline
#endif

namespace lrp {

LRP_CVT_FN uint64_t cvt_f64_bits(double x) {
#if defined(__CUDA_ARCH__)
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t b;
  memcpy(&b, &x, sizeof b);
  return b;
#endif
}

LRP_CVT_FN float cvt_f32_from_bits(uint32_t b) {
#if defined(__CUDA_ARCH__)
  return __uint_as_float(b);
#else
  float f;
  memcpy(&f, &b, sizeof f);
  return f;
#endif
}

LRP_CVT_FN float f64_to_f32_rn(double x) {
  const uint64_t b = cvt_f64_bits(x);
  const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
  const uint32_t sign = hi & 0x80000000u;
  const uint32_t ahi = hi & 0x7fffffffu;
  const uint32_t e = ahi >> 20;
  uint32_t r;
  if (e - 897u < 254u) {
    // e in [897, 1150]: FP32 biased exponent e - 896 in [1, 254].  Rebias,
    // keep the top 23 fraction bits; the 29 dropped bits decide the rounding.
    // A carry out of the fraction steps the exponent (to infinity above 254).
    r = ((ahi - (896u << 20)) << 3) | (lo >> 29);
    const uint32_t rest = lo & 0x1fffffffu;
    const uint32_t half = 0x10000000u;
    r += (rest > half || (rest == half && (r & 1u))) ? 1u : 0u;
  } else if (e >= 1151u) {
    if (e == 2047u) return (float)x;  // infinity or NaN: the hardware conversion
    r = 0x7f800000u;                  // |x| >= 2^128 rounds to infinity
  } else if (e >= 873u) {
    // FP32 subnormal (or the smallest normal after rounding): |x| = M 2^(e - 1075)
    // with the 53-bit significand M; in units of 2^-149 that is M / 2^(926 - e).
    const uint64_t M = (b & 0x000fffffffffffffull) | 0x0010000000000000ull;
    const uint32_t sh = 926u - e;  // 30 .. 53
    uint32_t q = (uint32_t)(M >> sh);
    const uint64_t rem = M & ((1ull << sh) - 1ull);
    const uint64_t half = 1ull << (sh - 1u);
    q += (rem > half || (rem == half && (q & 1u))) ? 1u : 0u;
    r = q;
  } else {
    r = 0u;  // |x| < 2^-150 (FP64 zeros and subnormals included): signed zero
  }
  return cvt_f32_from_bits(sign | r);
}

LRP_CVT_FN double cvt_f64_from_bits(uint64_t b) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double((long long)b);
#else
  double d;
  memcpy(&d, &b, sizeof d);
  return d;
#endif
}

LRP_CVT_FN uint32_t cvt_f32_bits(float f) {
#if defined(__CUDA_ARCH__)
  return __float_as_uint(f);
#else
  uint32_t b;
  memcpy(&b, &f, sizeof b);
  return b;
#endif
}

LRP_CVT_FN int cvt_clz32(uint32_t v) {  // v != 0
#if defined(__CUDA_ARCH__)
  return __clz((int)v);
#else
  int z = 0;
  while (!(v & 0x80000000u)) {
    v <<= 1;
    ++z;
  }
  return z;
#endif
}

// FP32 -> FP64 (exact for every finite value) on the integer pipe; infinities
// and NaNs take the hardware conversion.
LRP_CVT_FN double f32_to_f64(float f) {
  const uint32_t b = cvt_f32_bits(f);
  const uint64_t sign = (uint64_t)(b & 0x80000000u) << 32;
  const uint32_t a = b & 0x7fffffffu;
  const uint32_t e = a >> 23;
  if (e - 1u < 254u) {
    // normal: biased exponent e + 896, the 23 fraction bits at the top of 52
    return cvt_f64_from_bits(sign | (((uint64_t)a + (896ull << 23)) << 29));
  }
  if (e == 255u) return (double)f;
  if (a == 0u) return cvt_f64_from_bits(sign);
  // FP32 subnormal a 2^-149: normalise the fraction so that its leading one
  // sits at bit 23; the value is then (a << sh) 2^(-126 - sh - 23)
  const int sh = cvt_clz32(a) - 8;
  const uint64_t frac = (uint64_t)((a << sh) & 0x007fffffu) << 29;
  return cvt_f64_from_bits(sign | ((uint64_t)(897 - sh) << 52) | frac);
}

}  // namespace lrp

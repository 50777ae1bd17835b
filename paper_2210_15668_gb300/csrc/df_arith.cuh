// Double-float ("float-float") arithmetic on the FP32 pipe, for the FP64 outer
// residual of the mixed-precision form.  A value is the unevaluated sum h + l of
// two floats, about 48 significant bits.  GB300 executes FP64 at 1/58 of its FP32
// rate, so a stencil in double-float costs less than the same stencil in FP64.
//
// Error-free transformations, written from their published definitions:
//   TwoSum (Knuth, The Art of Computer Programming vol. 2, 4.2.2): s = fl(a + b)
//     and the exact rounding error e, a + b = s + e, for any a, b;
//   FastTwoSum (Dekker, Numer. Math. 18 (1971)): the same for |a| >= |b|, cheaper;
//   TwoProd by fused multiply-add: the exact error of p = fl(a b) is fma(a, b, -p).
// Double-float addition renormalises both the high and the low sums (the accurate
// form, needed here because the residual is a near-cancellation of b and A phi);
// multiplication adds the cross terms into the product's error.
#pragma once
#include <cuda_runtime.h>

namespace fx {
namespace dev {

struct df {
  float h, l;
};

__device__ __forceinline__ df df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}

__device__ __forceinline__ df df_fast_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}

__device__ __forceinline__ df df_add(df x, df y) {
  df s = df_two_sum(x.h, y.h);
  const df t = df_two_sum(x.l, y.l);
  s.l += t.h;
  s = df_fast_two_sum(s.h, s.l);
  s.l += t.l;
  return df_fast_two_sum(s.h, s.l);
}

// Addition that adds the low parts without their own TwoSum: its error is a few
// ulp of the low parts, i.e. about 2^-48 of the larger operand (not of the sum).
// The residual's tolerance is measured against its largest terms, so this is the
// form it uses.
__device__ __forceinline__ df df_add_fast(df x, df y) {
  df s = df_two_sum(x.h, y.h);
  s.l += x.l + y.l;
  return df_fast_two_sum(s.h, s.l);
}

__device__ __forceinline__ df df_neg(df x) { return {-x.h, -x.l}; }

__device__ __forceinline__ df df_mul(df x, df y) {
  const float p = x.h * y.h;
  float e = fmaf(x.h, y.h, -p);
  e = fmaf(x.h, y.l, e);
  e = fmaf(x.l, y.h, e);
  return df_fast_two_sum(p, e);
}

// An FP64 value as h + l with integer operations only (the FP64 -> FP32 conversion
// instruction runs on the FP64 pipe): h keeps the sign, the exponent and the top 23
// stored mantissa bits (truncated), l the next 24 of the remaining 29 (truncated),
// so h + l equals x to 2^-47 relative.  |x| < 2^-63 becomes zero (the scaled
// potentials and right-hand sides are many orders above); values beyond the FP32
// range become infinite (with the NaN payload kept).
__device__ __forceinline__ df df_from_double(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(u >> 32) & 0x80000000u;
  const int e = (int)((u >> 52) & 0x7ff);
  const unsigned mh = (unsigned)(u >> 29) & 0x7fffffu;
  if (e < 960) return {__uint_as_float(sign), 0.0f};
  if (e - 896 >= 255) return {__uint_as_float(sign | 0x7f800000u | mh), 0.0f};
  const float h = __uint_as_float(sign | ((unsigned)(e - 896) << 23) | mh);
  const unsigned r = (unsigned)u & 0x1fffffffu;         // the 29 bits below h's mantissa
  if (r == 0u) return {h, 0.0f};
  const int nb = 32 - __clz(r);                          // significant bits of r
  const unsigned m = nb > 24 ? r >> (nb - 24) : r << (24 - nb);
  // r 2^(e - 1075) = 1.m 2^(nb - 1 + e - 1075): biased FP32 exponent nb + e - 949 >= 12
  return {h, __uint_as_float(sign | ((unsigned)(nb + e - 949) << 23) | (m & 0x7fffffu))};
}

}  // namespace dev
}  // namespace fx

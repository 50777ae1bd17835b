// e^{+u} and e^{-u} of one argument, for the Boltzmann carrier densities
// n = n0 e^{phi/V_T}, p = p0 e^{-phi/V_T} of a semiconductor cell (Sec. II, the
// carrier model of the Poisson right-hand side).  Both come from one argument
// reduction, table-driven after Tang (ACM TOMS 15(2), 1989):
//
//   u = k ln2/64 + r,  k = round(64 u / ln2) = 64 q + j (0 <= j < 64),  |r| <= ln2/128,
//   e^{+u} = 2^{q}  T+[j] (1 + (e^{r} - 1)),   e^{-u} = 2^{-q} T-[j] (1 + (e^{-r} - 1)),
//
// T+-[j] = 2^{+-j/64} (nearest doubles, exp_table.cuh).  k is read from the low
// word of u 64/ln2 + 1.5 2^52; r = u - k ln2/64 with ln2/64 split in two parts
// (Cody and Waite) so that k ln2/64 is subtracted to well below one ulp of r.
// With E = r^2/2 + r^4/24 and O = r + r^3/6 + r^5/120 (Taylor series; the first
// dropped term is below 4e-17 relative for |r| <= ln2/128),
// e^{+-r} - 1 = E +- O, and each result is one final fma(s, E +- O, s).  Error
// at most about 1.3 ulp over |u| < 700; larger |u| (and NaN) take the library
// exponential, so overflow and underflow behave as exp() does.
#pragma once
#include "df_arith.cuh"
#include "exp_table.cuh"

namespace fx {

__device__ __forceinline__ double scale_pow2(double x, int q) {
  // x * 2^q for a normal x whose result stays normal: add q to the exponent field
  return __hiloint2double(__double2hiint(x) + q * (1 << 20), __double2loint(x));
}

__device__ __forceinline__ void exp_pm(double u, double& ep, double& em) {
  if (!(fabs(u) < 700.0)) {
    ep = exp(u);
    em = exp(-u);
    return;
  }
  const double shift = 0x1.8p52;
  const double t = fma(u, kExpInvL, shift);
  const double kd = t - shift;
  const int k = __double2loint(t);
  double r = fma(-kd, kExpLhi, u);
  r = fma(-kd, kExpLlo, r);
  const double r2 = r * r;
  const double E = r2 * fma(r2, 1.0 / 24.0, 0.5);
  const double O = fma(r * r2, fma(r2, 1.0 / 120.0, 1.0 / 6.0), r);
  const double2 tj = __ldg(&kExpTab[k & ((1 << kExpTabBits) - 1)]);
  const int q = k >> kExpTabBits;
  const double sp = scale_pow2(tj.x, q);
  const double sm = scale_pow2(tj.y, -q);
  ep = fma(sp, E + O, sp);
  em = fma(sm, E - O, sm);
}

// The same pair in double-float arithmetic on the FP32 pipe, for |u.h| <= kExpDFMax
// (callers take exp_pm beyond).  The reduction r = u - k ln2/64 uses ln2/64 =
// C1 + C2 + C3 + C4 with C1..C3 of 11 significant bits, so k C1, k C2, k C3 are
// exact for |k| < 2^13 and C4's product is kept exactly (two-product); r carries
// about 2^-60 absolute error.  e^{+-r} - 1 = E +- O with E = r^2/2 + r^4/24 and O =
// r + r^3/6 + r^5/120 (r^2, r^3 and r^3/6 as pairs, the two small terms in FP32;
// the first dropped terms are below 4e-17).  The results are the pairs
// 2^{+-q} T+-[j] (1 + (E +- O)) from the float-pair table, scaled by exact powers of
// two; both keep about 2^-47 relative accuracy while they stay normal floats.
constexpr float kExpDFMax = 70.0f;

__device__ __forceinline__ dev::df df_two_prod(float a, float b) {
  const float p = a * b;
  return {p, fmaf(a, b, -p)};
}

__device__ __forceinline__ void exp_pm_df(dev::df u, dev::df& ep, dev::df& em) {
  using dev::df;
  using dev::df_add;
  using dev::df_mul;
  const float kf = rintf(u.h * kExpInvLf);
  const int k = (int)kf;
  const float t1 = u.h - kf * kExpC1f;                       // exact (Sterbenz; k C1 exact)
  df r = dev::df_two_sum(t1, -kf * kExpC2f);                  // k C2 exact
  r = df_add(r, df{-kf * kExpC3f, 0.0f});                     // k C3 exact
  r = df_add(r, df{u.l, 0.0f});
  const df k4 = df_two_prod(kf, kExpC4f);
  r = df_add(r, df{-k4.h, -k4.l});
  const df r2 = df_mul(r, r);
  const df r3 = df_mul(r2, r);
  const float r4 = r2.h * r2.h;
  const df E = df_add(df{0.5f * r2.h, 0.5f * r2.l}, df{r4 * (1.0f / 24.0f), 0.0f});
  const df O = df_add(df_add(r, df_mul(r3, df{kSixthHf, kSixthLf})), df{r3.h * r2.h * (1.0f / 120.0f), 0.0f});
  const float4 tj = __ldg(&kExpTabDF[k & ((1 << kExpTabBits) - 1)]);
  const int q = k >> kExpTabBits;                              // floor(k / 64)
  const float sp = __int_as_float((127 + q) << 23), sm = __int_as_float((127 - q) << 23);
  const df Tp{tj.x * sp, tj.y * sp}, Tm{tj.z * sm, tj.w * sm};
  ep = df_add(Tp, df_mul(Tp, df_add(E, O)));
  em = df_add(Tm, df_mul(Tm, df_add(E, df{-O.h, -O.l})));
}

}  // namespace fx

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

}  // namespace fx

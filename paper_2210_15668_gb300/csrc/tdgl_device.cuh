// Per-column device functions of the fused TDGL update (Eq. TDGL2) and the
// Poisson right-hand side, shared by tdgl.cu and the persistent batched engine.
// See tdgl.cu for the method.
#pragma once
#include <cuda_runtime.h>

#include "ferrox_internal.cuh"

namespace fx {
namespace dev {

__device__ __forceinline__ double landau(double a, double b, double g, double P) {
  const double P2 = P * P;
  return P * fma(P2, fma(g, P2, b), a);
}

// z component of the force at plane k of column (i, j)
__device__ __forceinline__ double force_z(const TDGLArgs& a, const PlaneTDGL& pt,
                                          const PlaneTDGL* planes, const double* Pz,
                                          const double* phi, long long t, int k, int i, int j,
                                          int im, int ip, int jm, int jp, double v_bot,
                                          double v_top) {
  const long long plane = (long long)a.nx * a.ny;
  const double P = Pz[t];
  const double lat = (Pz[t - i + im] + Pz[t - i + ip]) +
                     (Pz[t + (long long)(jm - j) * a.nx] + Pz[t + (long long)(jp - j) * a.nx]);
  const bool fe_dn = k > 0 && __ldg(&planes[k - 1].fe);
  const bool fe_up = k < a.nz - 1 && __ldg(&planes[k + 1].fe);
  const double Pdn = fe_dn ? Pz[t - plane] : 0.0;
  const double Pup = fe_up ? Pz[t + plane] : 0.0;
  const double ph = phi[t];
  double phif_dn, phif_up;
  if (k == 0) {
    phif_dn = v_bot;
  } else {
    phif_dn = fma(pt.fw_L, phi[t - plane], pt.fw_R * ph) - pt.fpc * (P - Pdn);
  }
  if (k == a.nz - 1) {
    phif_up = v_top;
  } else {
    const PlaneTDGL pu = ldg_struct(planes + k + 1);
    phif_up = fma(pu.fw_L, ph, pu.fw_R * phi[t + plane]) - pu.fpc * (Pup - P);
  }
  const double lap = fma(-4.0, P, lat) * a.inv_h2;
  const double d2z = fma(pt.wz_dn, Pdn, fma(pt.wz_c, P, pt.wz_up * Pup));
  double dF = landau(pt.alpha, pt.beta, pt.gamma, P);
  dF = fma(-pt.g44, lap, dF);
  dF = fma(-pt.g11, d2z, dF);
  dF = fma(phif_up - phif_dn, a.inv_h, dF);
  return -pt.Gamma * dF;
}

// in-plane component (3-component model): own Landau polynomial and dPhi/dx
// from in-plane face potentials (equal permittivity on both sides of the face)
__device__ __forceinline__ double force_xy(const TDGLArgs& a, const PlaneTDGL& pt,
                                           const PlaneTDGL* planes, const double* Pc,
                                           const double* phi, long long t, int k, int i, int j,
                                           int im, int ip, int jm, int jp, int comp,
                                           double inv_eps_abs) {
  const long long plane = (long long)a.nx * a.ny;
  const double P = Pc[t];
  const long long tm = comp == 0 ? t - i + im : t + (long long)(jm - j) * a.nx;
  const long long tp = comp == 0 ? t - i + ip : t + (long long)(jp - j) * a.nx;
  const double lat = (Pc[t - i + im] + Pc[t - i + ip]) +
                     (Pc[t + (long long)(jm - j) * a.nx] + Pc[t + (long long)(jp - j) * a.nx]);
  const bool fe_dn = k > 0 && __ldg(&planes[k - 1].fe);
  const bool fe_up = k < a.nz - 1 && __ldg(&planes[k + 1].fe);
  const double Pdn = fe_dn ? Pc[t - plane] : 0.0;
  const double Pup = fe_up ? Pc[t + plane] : 0.0;
  const double lap = fma(-4.0, P, lat) * a.inv_h2;
  const double d2z = fma(pt.wz_dn, Pdn, fma(pt.wz_c, P, pt.wz_up * Pup));
  // (Phi_f(+) - Phi_f(-))/h = (phi_p - phi_m)/(2h) - (P_p - 2P + P_m)/(4 eps)
  const double dphi = 0.5 * (phi[tp] - phi[tm]) * a.inv_h -
                      0.25 * (Pc[tp] - 2.0 * P + Pc[tm]) * inv_eps_abs;
  double dF = landau(pt.alpha_xy, pt.beta_xy, pt.gamma_xy, P);
  dF = fma(-pt.g44, lap, dF);
  dF = fma(-pt.g11, d2z, dF);
  dF += dphi;
  return -pt.Gamma * dF;
}

__device__ __forceinline__ double advance(const TDGLArgs& a, long long idx, double f) {
  if (a.mode == 0) return a.P_in[idx] + a.dt * f;
  if (a.mode == 1) {
    a.F_store[idx] = f;
    return a.P_in[idx] + a.dt * f;
  }
  return a.P_base[idx] + 0.5 * a.dt * (a.F_store[idx] + f);
}

__device__ __forceinline__ double rhs_value(const TDGLArgs& a, const PlaneTDGL* planes, int k,
                                            double pn_dn, double pn, double pn_up, double v_bot,
                                            double v_top) {
  const double Pf_dn =
      (k == 0) ? pn : fma(__ldg(&planes[k].fw_R), pn_dn, __ldg(&planes[k].fw_L) * pn);
  const double Pf_up = (k == a.nz - 1)
                           ? pn
                           : fma(__ldg(&planes[k + 1].fw_R), pn, __ldg(&planes[k + 1].fw_L) * pn_up);
  double b = -(Pf_up - Pf_dn) * a.b_scale;
  if (k == 0) b = fma(__ldg(&planes[0].lift), v_bot, b);
  if (k == a.nz - 1) b = fma(__ldg(&planes[a.nz - 1].lift), v_top, b);
  return b;
}

// One (x, y) column of the TDGL update: march up the dynamic planes, write the
// new P of the FE planes and (uniaxial) the right-hand side b of every dynamic plane.
__device__ __forceinline__ void tdgl_column(const TDGLArgs& a, int i, int j) {
  const int im = (i == 0) ? a.nx - 1 : i - 1, ip = (i == a.nx - 1) ? 0 : i + 1;
  const int jm = (j == 0) ? a.ny - 1 : j - 1, jp = (j == a.ny - 1) ? 0 : j + 1;
  const long long plane = (long long)a.nx * a.ny;
  const long long N = plane * a.nz;
  const long long col = (long long)j * a.nx + i;
  const double v_bot = a.params->v_bot, v_top = a.params->v_top;
  const PlaneTDGL* planes = a.planes;
  const double* Pz_in = a.P_in + (long long)(a.ncomp - 1) * N;
  // ring of new P_z values at planes k-1, k (b of plane k-1 is emitted once P(k) is known)
  double pn_m2 = 0.0, pn_m1 = 0.0;
  for (int k = a.kd_lo; k <= a.kd_hi + 1; ++k) {
    double pn = 0.0;
    if (k <= a.kd_hi) {
      const PlaneTDGL pt = ldg_struct(planes + k);
      if (pt.fe && a.mode == 3) {
        pn = Pz_in[k * plane + col];          // right-hand side of the current P only
      } else if (pt.fe) {
        const long long t = k * plane + col;
        if (a.ncomp == 3) {
          const double inv_eps_abs = 1.0 / (8.8541878128e-12 * pt.eps_r);
          for (int c = 0; c < 2; ++c) {
            const double* Pc = a.P_in + (long long)c * N;
            const double f =
                force_xy(a, pt, planes, Pc, a.phi, t, k, i, j, im, ip, jm, jp, c, inv_eps_abs);
            a.P_out[c * N + t] = advance(a, c * N + t, f);
          }
        }
        const double f = force_z(a, pt, planes, Pz_in, a.phi, t, k, i, j, im, ip, jm, jp, v_bot, v_top);
        const long long zi = (long long)(a.ncomp - 1) * N + t;
        pn = advance(a, zi, f);
        a.P_out[zi] = pn;
      }
    }
    if (a.ncomp == 1 && k - 1 >= a.kd_lo) {
      a.b[(k - 1) * plane + col] = rhs_value(a, planes, k - 1, pn_m2, pn_m1, pn, v_bot, v_top);
    }
    pn_m2 = pn_m1;
    pn_m1 = pn;
  }
}

}  // namespace dev
}  // namespace fx

// TDGL polarization update (Eq. TDGL2) fused with the Poisson right-hand side,
// and the charge diagnostics of the Results section.
//
// One thread owns one (x, y) column and marches up the planes that can carry
// polarization, so the new P of the planes below, at and above a cell is in
// registers when that cell's right-hand side  b = -div_h P_f + lift  is formed:
// the new polarization and b leave the kernel in one pass.  Lateral
// neighbours are read from the previous state (explicit scheme), which is why
// the new P goes to a separate array.
//
// Force (per ferroelectric cell, component c):
//   f = -Gamma [ alpha P + beta P^3 + gamma P^5 - g44 (d2x + d2y) P - g11 d2z P + dPhi/dx_c ]
// with the P boundary conditions folded into per-plane d2z weights (one-sided
// second-order stencil through the face value; Methods, P boundary conditions)
// and dPhi/dz from the two face potentials of the cell (flux-continuous
// interpolation across material interfaces, electrode value on electrode faces).
#include <cuda_runtime.h>

#include "ferrox_internal.cuh"

namespace fx {

namespace {

constexpr int kBX = 32, kBY = 8;

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
  const bool fe_dn = k > 0 && planes[k - 1].fe;
  const bool fe_up = k < a.nz - 1 && planes[k + 1].fe;
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
    const PlaneTDGL& pu = planes[k + 1];
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
  const bool fe_dn = k > 0 && planes[k - 1].fe;
  const bool fe_up = k < a.nz - 1 && planes[k + 1].fe;
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
  const double Pf_dn = (k == 0) ? pn : fma(planes[k].fw_R, pn_dn, planes[k].fw_L * pn);
  const double Pf_up =
      (k == a.nz - 1) ? pn : fma(planes[k + 1].fw_R, pn, planes[k + 1].fw_L * pn_up);
  double b = -(Pf_up - Pf_dn) * a.b_scale;
  if (k == 0) b = fma(planes[0].lift, v_bot, b);
  if (k == a.nz - 1) b = fma(planes[a.nz - 1].lift, v_top, b);
  return b;
}

__global__ void __launch_bounds__(kBX* kBY) tdgl_kernel(TDGLArgs a) {
  const int i = blockIdx.x * kBX + threadIdx.x;
  const int j = blockIdx.y * kBY + threadIdx.y;
  if (i >= a.nx || j >= a.ny) return;
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
      const PlaneTDGL& pt = planes[k];
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

// b on the dynamic planes from an updated 3-component P (needs new in-plane
// neighbours, hence its own pass): z faces as above plus the central
// difference of the in-plane face averages of P_x and P_y.
__global__ void __launch_bounds__(kBX* kBY) rhs3_kernel(TDGLArgs a, const double* P) {
  const int i = blockIdx.x * kBX + threadIdx.x;
  const int j = blockIdx.y * kBY + threadIdx.y;
  if (i >= a.nx || j >= a.ny) return;
  const int im = (i == 0) ? a.nx - 1 : i - 1, ip = (i == a.nx - 1) ? 0 : i + 1;
  const int jm = (j == 0) ? a.ny - 1 : j - 1, jp = (j == a.ny - 1) ? 0 : j + 1;
  const long long plane = (long long)a.nx * a.ny;
  const long long N = plane * a.nz;
  const long long col = (long long)j * a.nx + i;
  const double v_bot = a.params->v_bot, v_top = a.params->v_top;
  const double* Pz = P + 2 * N;
  for (int k = a.kd_lo; k <= a.kd_hi; ++k) {
    const long long t = k * plane + col;
    const bool fe = a.planes[k].fe;
    const double pn = fe ? Pz[t] : 0.0;
    const double pdn = (k > 0 && a.planes[k - 1].fe) ? Pz[t - plane] : 0.0;
    const double pup = (k < a.nz - 1 && a.planes[k + 1].fe) ? Pz[t + plane] : 0.0;
    double b = rhs_value(a, a.planes, k, pdn, pn, pup, v_bot, v_top);
    if (fe) {
      const double dpx = P[t - i + ip] - P[t - i + im];
      const double dpy = P[N + t + (long long)(jp - j) * a.nx] - P[N + t + (long long)(jm - j) * a.nx];
      b -= 0.5 * (dpx + dpy) * a.b_scale;
    }
    a.b[t] = b;
  }
}

// --- diagnostics ------------------------------------------------------------------------
constexpr int kChargeBlocks = 64;

__device__ __forceinline__ double wsum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(256) charge_kernel(ChargeArgs a) {
  const long long plane = (long long)a.nx * a.ny;
  const double v_bot = a.params->v_bot, v_top = a.params->v_top;
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  const int k = a.k_int;
  const bool fe_top = a.planes[a.nz - 1].fe, fe_bot = a.planes[0].fe;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < plane;
       c += (long long)gridDim.x * blockDim.x) {
    const double* phi = a.phi;
    double F, phif;
    if (k > 0) {
      const PlaneTDGL& pt = a.planes[k];
      const double pL = phi[(k - 1) * plane + c], pR = phi[k * plane + c];
      const double PL = a.planes[k - 1].fe ? a.P[(k - 1) * plane + c] : 0.0;
      const double PR = pt.fe ? a.P[k * plane + c] : 0.0;
      const double eh = 2.0 * a.eps_L * a.eps_R / (a.eps_L + a.eps_R);
      F = -eh * (pR - pL) / a.h + fma(pt.fw_R, PL, pt.fw_L * PR);
      phif = fma(pt.fw_L, pL, pt.fw_R * pR) - pt.fpc * (PR - PL);
    } else {
      const double P0 = fe_bot ? a.P[c] : 0.0;
      F = -a.eps_bot * (phi[c] - v_bot) / (0.5 * a.h) + P0;
      phif = v_bot;
    }
    const double Pt = fe_top ? a.P[(a.nz - 1) * plane + c] : 0.0;
    const double Pb = fe_bot ? a.P[c] : 0.0;
    const double Ft = -a.eps_top * (v_top - phi[(a.nz - 1) * plane + c]) / (0.5 * a.h) + Pt;
    const double Fb = -a.eps_bot * (phi[c] - v_bot) / (0.5 * a.h) + Pb;
    s[0] += F; s[1] += phif; s[2] += Ft; s[3] += Fb;
  }
  __shared__ double sh[4][8];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  for (int q = 0; q < 4; ++q) {
    const double v = wsum(s[q]);
    if (l == 0) sh[q][w] = v;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double v = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) v += sh[threadIdx.x][q];
    a.partials[threadIdx.x * kChargeBlocks + blockIdx.x] = v;
  }
}

__global__ void charge_finalize(const double* partials, double* out) {
  if (threadIdx.x < 4) {
    double v = 0.0;
    for (int b = 0; b < kChargeBlocks; ++b) v += partials[threadIdx.x * kChargeBlocks + b];
    out[threadIdx.x] = v;
  }
}

__global__ void set_params_kernel(DevParams* p, double v_bot, double v_top) {
  p->v_bot = v_bot;
  p->v_top = v_top;
}

__global__ void stats_step_kernel(DevStats* st, int n, int launches) {
  st->steps += n;
  st->launches += launches;
}

}  // namespace

void launch_tdgl(const TDGLArgs& a, cudaStream_t s) {
  dim3 block(kBX, kBY);
  dim3 grid((a.nx + kBX - 1) / kBX, (a.ny + kBY - 1) / kBY);
  if (a.mode == 3 && a.ncomp == 3) {
    rhs3_kernel<<<grid, block, 0, s>>>(a, a.P_in);
    return;
  }
  tdgl_kernel<<<grid, block, 0, s>>>(a);
  if (a.ncomp == 3) rhs3_kernel<<<grid, block, 0, s>>>(a, a.P_out);
}

void launch_charge(const ChargeArgs& a, cudaStream_t s) {
  charge_kernel<<<kChargeBlocks, 256, 0, s>>>(a);
  charge_finalize<<<1, 32, 0, s>>>(a.partials, a.out);
}

void launch_set_params(DevParams* p, double v_bot, double v_top, cudaStream_t s) {
  set_params_kernel<<<1, 1, 0, s>>>(p, v_bot, v_top);
}

void launch_stats_step(DevStats* st, int nsteps, int launches, cudaStream_t s) {
  stats_step_kernel<<<1, 1, 0, s>>>(st, nsteps, launches);
}

}  // namespace fx

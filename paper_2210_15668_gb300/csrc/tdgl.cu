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
#include "tdgl_device.cuh"

namespace fx {

namespace {

constexpr int kBX = 32, kBY = 8;
using namespace dev;

__global__ void __launch_bounds__(kBX* kBY) tdgl_kernel(TDGLArgs a) {
  pdl_enter();
  const int i = blockIdx.x * kBX + threadIdx.x;
  const int j = blockIdx.y * kBY + threadIdx.y;
  if (i >= a.nx || j >= a.ny) return;
  tdgl_column(a, i, j);
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

// phi <- 2 phi - phi_prev, phi_prev <- phi (initial guess of the next solve)
__global__ void __launch_bounds__(256) extrapolate_kernel(double* __restrict__ phi,
                                                          double* __restrict__ prev, long long n) {
  pdl_enter();
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const double v = phi[t];
    phi[t] = fma(2.0, v, -prev[t]);
    prev[t] = v;
  }
}

__global__ void set_params_kernel(DevParams* p, double v_bot, double v_top) {
  p->v_bot = v_bot;
  p->v_top = v_top;
}

// The electrode lift of the boundary planes whose right-hand side no TDGL update
// writes (b of the other static planes stays zero), so that b holds the whole
// right-hand side for the direct FP64 form's sweeps on phi.
__global__ void static_b_kernel(double* b, const PlaneTDGL* planes, const DevParams* prm, int nx,
                                int ny, int nz) {
  const long long plane = (long long)nx * ny;
  const int side = blockIdx.y;               // 0: bottom plane, 1: top plane
  const int k = side == 0 ? 0 : nz - 1;
  if (side == 1 && nz == 1) return;          // one plane: written once, both lifts
  const PlaneTDGL& pt = planes[k];
  if (pt.b_dyn) return;
  double v = 0.0;
  if (k == 0) v += pt.lift * prm->v_bot;
  if (k == nz - 1) v += pt.lift * prm->v_top;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < plane;
       t += (long long)gridDim.x * blockDim.x)
    b[k * plane + t] = v;
}

// Holds the stream for a bounded number of SM clock cycles (the profiler queues a
// batch of launches behind it so that they then run back to back).
__global__ void delay_kernel(long long cycles) {
  const long long t0 = clock64();
  while (clock64() - t0 < cycles) {
  }
}

__global__ void stats_step_kernel(DevStats* st, int n, int launches) {
  pdl_enter();
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
  launch_k(tdgl_kernel, grid, block, 0, s, a);
  if (a.ncomp == 3) rhs3_kernel<<<grid, block, 0, s>>>(a, a.P_out);
}

void launch_charge(const ChargeArgs& a, cudaStream_t s) {
  charge_kernel<<<kChargeBlocks, 256, 0, s>>>(a);
  charge_finalize<<<1, 32, 0, s>>>(a.partials, a.out);
}

void launch_extrapolate(double* phi, double* prev, long long n, cudaStream_t s) {
  long long b = (n + 255) / 256;
  if (b > 152LL * 16) b = 152LL * 16;
  launch_k(extrapolate_kernel, dim3((int)b), dim3(256), 0, s, phi, prev, n);
}

void launch_set_params(DevParams* p, double v_bot, double v_top, cudaStream_t s) {
  set_params_kernel<<<1, 1, 0, s>>>(p, v_bot, v_top);
}

void launch_static_b(double* b, const PlaneTDGL* planes, const DevParams* prm, int nx, int ny,
                     int nz, cudaStream_t s) {
  long long blocks = ((long long)nx * ny + 255) / 256;
  if (blocks > 152) blocks = 152;
  static_b_kernel<<<dim3((int)blocks, 2), 256, 0, s>>>(b, planes, prm, nx, ny, nz);
}

void launch_delay(long long cycles, cudaStream_t s) { delay_kernel<<<1, 1, 0, s>>>(cycles); }

void launch_stats_step(DevStats* st, int nsteps, int launches, cudaStream_t s) {
  launch_k(stats_step_kernel, dim3(1), dim3(1), 0, s, st, nsteps, launches);
}

}  // namespace fx

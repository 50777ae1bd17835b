// Geometric multigrid for the variable-permittivity 7-point operator and the
// FP64 outer (defect-correction / Newton) residual.
//
// The paper solves its Poisson problem with AMReX's geometric multigrid to a
// residual threshold (Methods, "Numerical Approach and Implementation"); this
// is an independent cell-centred multigrid written for one GPU:
//   * the outer loop works in FP64: r = b + rho(phi) - A phi, the Newton shift
//     s = -d rho/d phi in semiconductor cells, and the norms that decide
//     convergence (||r|| <= tol max(||b||, ||rho||)), all in one kernel whose last
//     block sums the per-block partials in a fixed order (deterministic);
//   * one V-cycle on (A + diag s) e = r in precision T (double, or float in the
//     mixed form): red-black Gauss-Seidel smoothing, residual fused with
//     full-weighting (8-child mean) restriction, trilinear (or constant)
//     prolongation fused with the correction, and the levels at or below
//     kTailMaxCells handled by one CTA in a single launch;
//   * phi += e in FP64 (clamped in semiconductor stacks: damped Newton).
#include <cuda_runtime.h>
#include <math.h>

#include "ferrox_internal.cuh"

namespace fx {

namespace {

__device__ __forceinline__ long long lidx(const LevelDesc& L, int i, int j, int k) {
  return L.off + ((long long)k * L.ny + j) * L.nx + i;
}

// (r + sum of couplings * neighbours) of one cell; the Gauss-Seidel numerator.
template <typename T>
__device__ __forceinline__ T gs_numerator(const T* e, const T* r,
                                          const PlaneCoef<T>& c, const LevelDesc& L, int i, int j,
                                          int k, long long id) {
  const int im = (i == 0) ? L.nx - 1 : i - 1;
  const int ip = (i == L.nx - 1) ? 0 : i + 1;
  const int jm = (j == 0) ? L.ny - 1 : j - 1;
  const int jp = (j == L.ny - 1) ? 0 : j + 1;
  const long long row = id - i;
  const long long plane = (long long)L.nx * L.ny;
  T sx = e[row + im] + e[row + ip];
  T sy = e[id + (long long)(jm - j) * L.nx] + e[id + (long long)(jp - j) * L.nx];
  T ed = (k > 0) ? e[id - plane] : T(0);
  T eu = (k < L.nz - 1) ? e[id + plane] : T(0);
  T acc = r[id];
  acc = fma(c.cx, sx, acc);
  acc = fma(c.cy, sy, acc);
  acc = fma(c.czlo, ed, acc);
  acc = fma(c.czhi, eu, acc);
  return acc;
}

template <typename T>
__device__ __forceinline__ void smooth_cell(const MGArgs<T>& a, const LevelDesc& L, int i, int j,
                                            int k, int color, int zero_init) {
  const PlaneCoef<T> c = a.coef[L.coef_off + k];
  const long long id = lidx(L, i, j, k);
  if (zero_init) {
    // first red half-sweep from e = 0: e_red = r / diag, and black cells start at 0
    T d = c.has_s ? T(1) / (c.diag + a.s[id]) : c.invdiag;
    a.e[id] = a.r[id] * d;
    (void)color;
    return;
  }
  T num = gs_numerator(a.e, a.r, c, L, i, j, k, id);
  a.e[id] = c.has_s ? num / (c.diag + a.s[id]) : num * c.invdiag;
}

// colour sweep over a level; t enumerates (half-row position, row, plane)
template <typename T>
__device__ __forceinline__ void smooth_item(const MGArgs<T>& a, const LevelDesc& L, long long t,
                                            int color, int zero_init) {
  const int hx = (L.nx + 1) >> 1;
  const int ip = (int)(t % hx);
  const long long rest = t / hx;
  const int j = (int)(rest % L.ny);
  const int k = (int)(rest / L.ny);
  const int par = (j + k + color) & 1;
  const int i = 2 * ip + par;
  if (i < L.nx) smooth_cell(a, L, i, j, k, color, zero_init);
  if (zero_init) {
    const int i2 = 2 * ip + (par ^ 1);
    if (i2 < L.nx) a.e[lidx(L, i2, j, k)] = T(0);
  }
}

// residual of one fine cell: r - (A + s) e
template <typename T>
__device__ __forceinline__ T cell_residual(const MGArgs<T>& a, const LevelDesc& L, int i, int j,
                                           int k) {
  const PlaneCoef<T> c = a.coef[L.coef_off + k];
  const long long id = lidx(L, i, j, k);
  T num = gs_numerator(a.e, a.r, c, L, i, j, k, id);   // r + couplings * neighbours
  T d = c.has_s ? c.diag + a.s[id] : c.diag;
  return fma(-d, a.e[id], num);
}

template <typename T>
__device__ __forceinline__ void restrict_item(const MGArgs<T>& a, const LevelDesc& F,
                                              const LevelDesc& C, long long t) {
  const int I = (int)(t % C.nx);
  const long long rest = t / C.nx;
  const int J = (int)(rest % C.ny);
  const int K = (int)(rest / C.ny);
  const int nxc = F.crx ? 2 : 1, nyc = F.cry ? 2 : 1, nzc = F.crz ? 2 : 1;
  const int i0 = F.crx ? 2 * I : I, j0 = F.cry ? 2 * J : J, k0 = F.crz ? 2 * K : K;
  T sum = T(0), ssum = T(0);
  for (int dk = 0; dk < nzc; ++dk)
    for (int dj = 0; dj < nyc; ++dj)
      for (int di = 0; di < nxc; ++di) {
        sum += cell_residual(a, F, i0 + di, j0 + dj, k0 + dk);
        if (a.s) ssum += a.s[lidx(F, i0 + di, j0 + dj, k0 + dk)];
      }
  const T inv = T(1) / T(nxc * nyc * nzc);
  const long long idc = lidx(C, I, J, K);
  a.r[idc] = sum * inv;
  if (a.s) a.s[idc] = ssum * inv;
}

template <typename T>
__device__ __forceinline__ void prolong_item(const MGArgs<T>& a, const LevelDesc& F,
                                             const LevelDesc& C, long long t, int constant) {
  const int i = (int)(t % F.nx);
  const long long rest = t / F.nx;
  const int j = (int)(rest % F.ny);
  const int k = (int)(rest / F.ny);
  const int I = F.crx ? (i >> 1) : i, J = F.cry ? (j >> 1) : j, K = F.crz ? (k >> 1) : k;
  const long long id = lidx(F, i, j, k);
  if (constant) {
    a.e[id] += a.e[lidx(C, I, J, K)];
    return;
  }
  // trilinear, cell-centred: weights 3/4 (own coarse cell) and 1/4 (the coarse
  // neighbour on the side of the fine cell) per coarsened direction
  int In = I, Jn = J, Kn = K;
  T wxo = T(1), wyo = T(1), wzo = T(1);
  T wxn = T(0), wyn = T(0), wzn = T(0);
  if (F.crx) {
    In = (i & 1) ? (I + 1 == C.nx ? 0 : I + 1) : (I == 0 ? C.nx - 1 : I - 1);
    wxo = T(0.75); wxn = T(0.25);
  }
  if (F.cry) {
    Jn = (j & 1) ? (J + 1 == C.ny ? 0 : J + 1) : (J == 0 ? C.ny - 1 : J - 1);
    wyo = T(0.75); wyn = T(0.25);
  }
  if (F.crz) {
    Kn = (k & 1) ? K + 1 : K - 1;
    wzo = T(0.75); wzn = T(0.25);
    if (Kn < 0 || Kn >= C.nz) {   // electrode: ghost value -e (zero correction on the face)
      Kn = K; wzo = T(0.5); wzn = T(0);
    }
  }
  const T* E = a.e;
  T v0 = wxo * E[lidx(C, I, J, K)] + wxn * E[lidx(C, In, J, K)];
  T v1 = wxo * E[lidx(C, I, Jn, K)] + wxn * E[lidx(C, In, Jn, K)];
  T lo = wyo * v0 + wyn * v1;
  T v2 = wxo * E[lidx(C, I, J, Kn)] + wxn * E[lidx(C, In, J, Kn)];
  T v3 = wxo * E[lidx(C, I, Jn, Kn)] + wxn * E[lidx(C, In, Jn, Kn)];
  T hi = wyo * v2 + wyn * v3;
  a.e[id] += wzo * lo + wzn * hi;
}

template <typename T>
__global__ void __launch_bounds__(256) smooth_kernel(MGArgs<T> a, LevelDesc L, int color,
                                                     int zero_init) {
  const long long total = (long long)((L.nx + 1) >> 1) * L.ny * L.nz;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x)
    smooth_item(a, L, t, color, zero_init);
}

template <typename T>
__global__ void __launch_bounds__(256) restrict_kernel(MGArgs<T> a, LevelDesc F, LevelDesc C) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < C.ncell;
       t += (long long)gridDim.x * blockDim.x)
    restrict_item(a, F, C, t);
}

template <typename T>
__global__ void __launch_bounds__(256) prolong_kernel(MGArgs<T> a, LevelDesc F, LevelDesc C,
                                                      int constant) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < F.ncell;
       t += (long long)gridDim.x * blockDim.x)
    prolong_item(a, F, C, t, constant);
}

// All levels l_first..l_last in one CTA: a complete V-cycle below l_first
// (pre-smoothing, restriction, bottom sweeps, prolongation, post-smoothing),
// with block barriers between the phases.
template <typename T>
__device__ void tail_smooth(const MGArgs<T>& a, const LevelDesc& L, int sweeps, int zero_first) {
  const long long half = (long long)((L.nx + 1) >> 1) * L.ny * L.nz;
  for (int sw = 0; sw < sweeps; ++sw)
    for (int color = 0; color < 2; ++color) {
      const int zi = (zero_first && sw == 0 && color == 0);
      for (long long t = threadIdx.x; t < half; t += blockDim.x) smooth_item(a, L, t, color, zi);
      __syncthreads();
    }
}

template <typename T>
__global__ void __launch_bounds__(kTailThreads) tail_kernel(MGArgs<T> a, int l_first, int l_last,
                                                            int nu1, int nu2, int bottom_sweeps,
                                                            int constant) {
  for (int l = l_first; l < l_last; ++l) {
    const LevelDesc F = a.lv[l], C = a.lv[l + 1];
    tail_smooth(a, F, nu1, 1);
    for (long long t = threadIdx.x; t < C.ncell; t += blockDim.x) restrict_item(a, F, C, t);
    __syncthreads();
  }
  tail_smooth(a, a.lv[l_last], bottom_sweeps, 1);
  for (int l = l_last - 1; l >= l_first; --l) {
    const LevelDesc F = a.lv[l], C = a.lv[l + 1];
    for (long long t = threadIdx.x; t < F.ncell; t += blockDim.x) prolong_item(a, F, C, t, constant);
    __syncthreads();
    tail_smooth(a, F, nu2, 0);
  }
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block sum of three values; result valid in thread 0.
__device__ __forceinline__ void block_sum3(double& x, double& y, double& z) {
  __shared__ double sh[3][32];
  x = warp_sum(x); y = warp_sum(y); z = warp_sum(z);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { sh[0][w] = x; sh[1][w] = y; sh[2][w] = z; }
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  if (w == 0) {
    x = l < nw ? sh[0][l] : 0.0;
    y = l < nw ? sh[1][l] : 0.0;
    z = l < nw ? sh[2][l] : 0.0;
    x = warp_sum(x); y = warp_sum(y); z = warp_sum(z);
  }
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(kResidThreads) resid_kernel(ResidArgs a) {
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const long long plane = (long long)nx * ny;
  const long long total = plane * nz;
  const double v_bot = a.params->v_bot, v_top = a.params->v_top;
  T* r_out = static_cast<T*>(a.r_out);
  T* s_out = static_cast<T*>(a.s_out);
  double acc_r = 0.0, acc_b = 0.0, acc_rho = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % nx);
    const int j = (int)((t / nx) % ny);
    const int k = (int)(t / plane);
    const PlaneCoef<double> c = a.coef0[k];
    const PlaneTDGL& pt = a.planes[k];
    const int im = (i == 0) ? nx - 1 : i - 1, ip = (i == nx - 1) ? 0 : i + 1;
    const int jm = (j == 0) ? ny - 1 : j - 1, jp = (j == ny - 1) ? 0 : j + 1;
    const double* phi = a.phi;
    const double pc = phi[t];
    const double sx = phi[t - i + im] + phi[t - i + ip];
    const double sy = phi[t + (long long)(jm - j) * nx] + phi[t + (long long)(jp - j) * nx];
    const double pd = (k > 0) ? phi[t - plane] : 0.0;
    const double pu = (k < nz - 1) ? phi[t + plane] : 0.0;
    double off = c.cx * sx;
    off = fma(c.cy, sy, off);
    off = fma(c.czlo, pd, off);
    off = fma(c.czhi, pu, off);
    double bb;
    if (pt.b_dyn) {
      bb = a.b[t];
    } else {
      bb = 0.0;
      if (k == 0) bb += pt.lift * v_bot;
      if (k == nz - 1) bb += pt.lift * v_top;
    }
    double rho = 0.0, sh = 0.0;
    if (pt.sc) {
      const double u = pc * pt.inv_vt;
      const double n = pt.n0 * exp(u);
      const double p = pt.p0 * exp(-u);
      rho = pt.kq * (p - n + pt.Nnet);
      sh = pt.kq * (n + p) * pt.inv_vt;
    }
    const double r = (bb + rho) - fma(c.diag, pc, -off);
    r_out[t] = (T)r;
    if (s_out && pt.sc) s_out[t] = (T)sh;
    acc_r = fma(r, r, acc_r);
    acc_b = fma(bb, bb, acc_b);
    acc_rho = fma(rho, rho, acc_rho);
  }
  block_sum3(acc_r, acc_b, acc_rho);
  __shared__ bool last;
  if (threadIdx.x == 0) {
    a.partials[blockIdx.x] = acc_r;
    a.partials[gridDim.x + blockIdx.x] = acc_b;
    a.partials[2 * gridDim.x + blockIdx.x] = acc_rho;
    __threadfence();
    const unsigned int prev = atomicAdd(&a.stats->done_ctr, 1u);
    last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // fixed-order sum of the partials: thread t takes blocks t, t+256, ..., then a tree
  double sr = 0.0, sb = 0.0, sq = 0.0;
  const volatile double* P = a.partials;
  for (int q = threadIdx.x; q < (int)gridDim.x; q += blockDim.x) {
    sr += P[q];
    sb += P[gridDim.x + q];
    sq += P[2 * gridDim.x + q];
  }
  block_sum3(sr, sb, sq);
  if (threadIdx.x == 0) {
    DevStats* st = a.stats;
    st->done_ctr = 0;
    if (a.first) {
      st->solves += 1;
      st->cycles_this_solve = 0;
      st->zero_phi = 0;
      st->launches += 1;
    }
    const double rn = sqrt(sr);
    const double scale = fmax(sqrt(sb), sqrt(sq));
    int cond;
    if (!isfinite(rn) || !isfinite(scale)) {
      if (st->status == 0) st->status = FERROX_ENONFINITE;
      cond = 0;
    } else if (rn <= a.tol * scale) {
      cond = 0;
    } else if (st->cycles_this_solve >= a.max_cycles) {
      if (st->status == 0) st->status = FERROX_ENOCONV;
      cond = 0;
    } else {
      // scale == 0 with r != 0: b = 0 and rho(phi) = 0, whose solution is phi = 0
      if (scale == 0.0) st->zero_phi = 1;
      cond = 1;
    }
    if (cond) {
      st->cycles_this_solve += 1;
      st->cycles += 1;
      st->launches += a.launches_per_cycle;
    }
    st->last_cond = cond;
    st->last_cycles = st->cycles_this_solve;
    st->last_rnorm = rn;
    st->last_scale = scale;
    st->last_rel = scale > 0.0 ? rn / scale : (rn > 0.0 ? INFINITY : 0.0);
    if (a.set_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)a.cond_handle, cond);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) update_kernel(double* __restrict__ phi, const T* __restrict__ e0,
                                                     long long n, const DevStats* stats,
                                                     double clamp) {
  const bool zero = stats->zero_phi != 0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    if (zero) {
      phi[t] = 0.0;
    } else {
      const double d = (double)e0[t];
      phi[t] += fmin(fmax(d, -clamp), clamp);
    }
  }
}

int grid_for(long long work, int threads) {
  long long b = (work + threads - 1) / threads;
  const long long cap = 152LL * 16;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

template <typename T>
void launch_smooth(const MGArgs<T>& a, const LevelDesc& L, int color, int zero_init, cudaStream_t s) {
  const long long half = (long long)((L.nx + 1) >> 1) * L.ny * L.nz;
  smooth_kernel<T><<<grid_for(half, 256), 256, 0, s>>>(a, L, color, zero_init);
}

template <typename T>
void launch_restrict(const MGArgs<T>& a, const LevelDesc& F, const LevelDesc& C, cudaStream_t s) {
  restrict_kernel<T><<<grid_for(C.ncell, 256), 256, 0, s>>>(a, F, C);
}

template <typename T>
void launch_prolong(const MGArgs<T>& a, const LevelDesc& F, const LevelDesc& C, int constant,
                    cudaStream_t s) {
  prolong_kernel<T><<<grid_for(F.ncell, 256), 256, 0, s>>>(a, F, C, constant);
}

template <typename T>
void launch_tail(const MGArgs<T>& a, int l_first, int l_last, int nu1, int nu2, int bottom_sweeps,
                 int constant, cudaStream_t s) {
  tail_kernel<T><<<1, kTailThreads, 0, s>>>(a, l_first, l_last, nu1, nu2, bottom_sweeps, constant);
}

template <typename T>
void launch_resid(const ResidArgs& a, cudaStream_t s) {
  resid_kernel<T><<<kResidBlocks, kResidThreads, 0, s>>>(a);
}

template <typename T>
void launch_update(double* phi, const T* e0, long long n, const DevStats* stats, double clamp,
                   cudaStream_t s) {
  update_kernel<T><<<grid_for(n, 256), 256, 0, s>>>(phi, e0, n, stats, clamp);
}

#define FX_INST(T)                                                                              \
  template void launch_smooth<T>(const MGArgs<T>&, const LevelDesc&, int, int, cudaStream_t);   \
  template void launch_restrict<T>(const MGArgs<T>&, const LevelDesc&, const LevelDesc&,        \
                                   cudaStream_t);                                               \
  template void launch_prolong<T>(const MGArgs<T>&, const LevelDesc&, const LevelDesc&, int,    \
                                  cudaStream_t);                                                \
  template void launch_tail<T>(const MGArgs<T>&, int, int, int, int, int, int, cudaStream_t);   \
  template void launch_resid<T>(const ResidArgs&, cudaStream_t);                                \
  template void launch_update<T>(double*, const T*, long long, const DevStats*, double,         \
                                 cudaStream_t);
FX_INST(double)
FX_INST(float)
#undef FX_INST

}  // namespace fx

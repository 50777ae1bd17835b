// Geometric multigrid for the variable-permittivity 7-point operator and the
// FP64 outer (defect-correction / Newton) residual.
//
// The paper solves its Poisson problem with AMReX's geometric multigrid to a
// residual threshold (Methods, "Numerical Approach and Implementation"); this
// is an independent cell-centred multigrid written for one GPU:
//   * the outer loop works in FP64: r = b + rho(phi) - A phi, the Newton shift
//     s = -d rho/d phi in semiconductor cells, and the norms that decide
//     convergence (||r|| <= tol max(||b||, ||rho||)), all in one z-marching
//     kernel whose last block sums the per-block partials in a fixed order
//     (deterministic) and sets the CUDA-graph loop condition;
//   * one V-cycle on (A + diag s) e = r in precision T (double, or float in the
//     mixed form): red-black Gauss-Seidel colour sweeps, residual fused with
//     8-child-mean restriction, trilinear prolongation fused with the
//     correction (one thread per coarse cell, separable), and every level at or
//     below the tail size solved by one CTA in shared memory in one launch;
//   * phi += e in FP64 fused into the last fine-level black sweep (clamped in
//     semiconductor stacks: damped Newton).
// Launch grids are 3-D (x chunk, row, plane), so no kernel divides indices.
#include <cuda_runtime.h>
#include <math.h>

#include "ferrox_internal.cuh"
#include "mg_device.cuh"

namespace fx {

namespace {

using namespace dev;

// ---- multi-block kernels (3-D grids: x chunk, row chunk, plane) ----------------------

// zst (direct FP64 form, sweeps on phi itself): when the solve found b = 0 with
// no carrier charge (zero_phi), write the solution phi = 0 instead of relaxing
template <typename T>
__global__ void __launch_bounds__(256) smooth_kernel(MGArgs<T> a, LevelDesc L, int color,
                                                     int zero_init, Upd u, const DevStats* st,
                                                     const DevStats* zst) {
  pdl_enter();
  const int ip = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (ip >= ((L.nx + 1) >> 1) || j >= L.ny) return;
  if (zst && zst->zero_phi) {
    const int i = 2 * ip + ((j + k + color) & 1);
    if (i < L.nx) a.e[lidx(L, i, j, k)] = T(0);
    return;
  }
  if (u.phi) u.zero = st->zero_phi;
  smooth_pair(a, L, ip, j, k, color, zero_init, u);
}

// A plain colour sweep (no zero start, no fused update) with KZ planes per
// thread: the loads of all KZ cells are issued before their arithmetic, so each
// thread keeps KZ independent chains in flight.  Same operations in the same
// order as smooth_pair.
template <typename T, int KZ>
__global__ void __launch_bounds__(256) smooth_kz_kernel(MGArgs<T> a, LevelDesc L, int color,
                                                        const DevStats* zst) {
  pdl_enter();
  const int ip = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k0 = blockIdx.z * KZ;
  if (ip >= ((L.nx + 1) >> 1) || j >= L.ny) return;
  const bool zero = zst && zst->zero_phi;
  const int plane = L.nx * L.ny;
  const int dym = ((j == 0) ? L.ny - 1 : j - 1) - j, dyp = ((j == L.ny - 1) ? 0 : j + 1) - j;
  int ids[KZ];
  T v[KZ][7];   // r, x-, x+, y-, y+, z-, z+
  PlaneCoef<T> c[KZ];
#pragma unroll
  for (int q = 0; q < KZ; ++q) {
    const int k = k0 + q;
    const int i = 2 * ip + ((j + k + color) & 1);
    ids[q] = (k < L.nz && i < L.nx) ? lidx(L, i, j, k) : -1;
    if (ids[q] < 0 || zero) continue;
    const int id = ids[q];
    const int im = (i == 0) ? L.nx - 1 : i - 1;
    const int ipp = (i == L.nx - 1) ? 0 : i + 1;
    c[q] = ldg_struct(a.coef + L.coef_off + k);
    v[q][0] = a.r[id];
    v[q][1] = a.e[id - i + im];
    v[q][2] = a.e[id - i + ipp];
    v[q][3] = a.e[id + dym * L.nx];
    v[q][4] = a.e[id + dyp * L.nx];
    v[q][5] = (k > 0) ? a.e[id - plane] : T(0);
    v[q][6] = (k < L.nz - 1) ? a.e[id + plane] : T(0);
  }
#pragma unroll
  for (int q = 0; q < KZ; ++q) {
    const int id = ids[q];
    if (id < 0) continue;
    if (zero) {
      a.e[id] = T(0);
      continue;
    }
    T acc = v[q][0];
    acc = fma(c[q].cx, v[q][1] + v[q][2], acc);
    acc = fma(c[q].cy, v[q][3] + v[q][4], acc);
    acc = fma(c[q].czlo, v[q][5], acc);
    acc = fma(c[q].czhi, v[q][6], acc);
    a.e[id] = c[q].has_s ? acc / (c[q].diag + a.s[id]) : acc * c[q].invdiag;
  }
}

// ---- fused red-black sweep (one launch per full sweep, out of place) -------------------
// One red-black Gauss-Seidel sweep of a level (red cells, then black cells) in
// one launch, reading e_in and writing e_out.  A block owns a TX x TY x TZ tile.
// It stages e_in on the tile plus a two-cell halo and r on the tile plus a
// one-cell halo in shared memory, relaxes the red cells of the tile and of its
// one-cell halo (the halo's red values are recomputed from the same inputs and
// operations as in the block that owns those cells, so they are identical),
// relaxes the black cells of the tile against them, and writes both colours of
// the tile.  Red cells are (i + j + k) even, as in the colour sweeps.  Every
// cell sees the operations of smooth_pair in the same order, so one launch
// equals the red sweep followed by the black sweep bit for bit, while each
// array element is read and written once per full sweep instead of once per
// colour.  Lateral sizes must be even and at least the tile's (one periodic
// wrap covers the halo); z beyond the level is the zero of the correction
// equation's Dirichlet faces.  With zero_init the sweep starts from e = 0
// (e_in unused).  With u.phi set, phi += e of both colours (clamped) follows.
template <typename T>
struct RBArgs {
  const T* e_in;            // level-relative
  T* e_out;                 // level-relative
  const T* r;               // level-relative
  const T* s;               // level-relative Newton shift (null without SC)
  const PlaneCoef<T>* coef; // the level's planes
  int nx, ny, nz;
  int zero_init;
  Upd u;
  const DevStats* st;       // zero_phi flag for the fused update
};

template <typename T, int TX, int TY, int TZ>
__global__ void __launch_bounds__(256) smooth_rb_kernel(RBArgs<T> a) {
  pdl_enter();
  constexpr int EX = TX + 4, EY = TY + 4, EZ = TZ + 4, EN = EX * EY * EZ;
  constexpr int RX = TX + 2, RY = TY + 2, RZ = TZ + 2, RN = RX * RY * RZ;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PlaneCoef<T>* Cs = reinterpret_cast<PlaneCoef<T>*>(smem_raw);
  T* Es = reinterpret_cast<T*>(smem_raw + ((RZ * sizeof(PlaneCoef<T>) + 15) / 16) * 16);
  T* Rs = Es + (a.zero_init ? 0 : EN);
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * TZ;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int plane = nx * ny;
  // stage: e_in with a two-cell halo (zero outside 0..nz-1), r with a one-cell halo
  if (!a.zero_init) {
    for (int q = tid; q < EN; q += 256) {
      const int xx = q % EX, t = q / EX, yy = t % EY, zz = t / EY;
      int x = x0 - 2 + xx, y = y0 - 2 + yy;
      const int z = z0 - 2 + zz;
      x += x < 0 ? nx : 0; x -= x >= nx ? nx : 0;
      y += y < 0 ? ny : 0; y -= y >= ny ? ny : 0;
      Es[q] = (z >= 0 && z < nz) ? a.e_in[z * plane + y * nx + x] : T(0);
    }
  }
  for (int q = tid; q < RN; q += 256) {
    const int xx = q % RX, t = q / RX, yy = t % RY, zz = t / RY;
    int x = x0 - 1 + xx, y = y0 - 1 + yy;
    const int z = z0 - 1 + zz;
    x += x < 0 ? nx : 0; x -= x >= nx ? nx : 0;
    y += y < 0 ? ny : 0; y -= y >= ny ? ny : 0;
    Rs[q] = (z >= 0 && z < nz) ? a.r[z * plane + y * nx + x] : T(0);
  }
  if (tid < RZ) {
    const int z = z0 - 1 + tid;
    if (z >= 0 && z < nz) Cs[tid] = ldg_struct(a.coef + z);
  }
  __syncthreads();
  // red cells of the tile and its one-cell halo; Rs then holds the new red values
  for (int q = tid; q < RN; q += 256) {
    const int xx = q % RX, t = q / RX, yy = t % RY, zz = t / RY;
    int x = x0 - 1 + xx, y = y0 - 1 + yy;
    const int z = z0 - 1 + zz;
    if (z < 0 || z >= nz) continue;
    x += x < 0 ? nx : 0; x -= x >= nx ? nx : 0;
    y += y < 0 ? ny : 0; y -= y >= ny ? ny : 0;
    if ((x + y + z) & 1) continue;
    const PlaneCoef<T> c = Cs[zz];
    const int id = z * plane + y * nx + x;
    T ev;
    if (a.zero_init) {
      const T d = c.has_s ? T(1) / (c.diag + a.s[id]) : c.invdiag;
      ev = Rs[q] * d;
    } else {
      const int e = ((zz + 1) * EY + (yy + 1)) * EX + (xx + 1);
      T acc = Rs[q];
      acc = fma(c.cx, Es[e - 1] + Es[e + 1], acc);
      acc = fma(c.cy, Es[e - EX] + Es[e + EX], acc);
      acc = fma(c.czlo, Es[e - EX * EY], acc);
      acc = fma(c.czhi, Es[e + EX * EY], acc);
      ev = c.has_s ? acc / (c.diag + a.s[id]) : acc * c.invdiag;
    }
    Rs[q] = ev;
  }
  __syncthreads();
  // black cells of the tile against the new red values; both colours written out
  Upd u = a.u;
  if (u.phi) u.zero = a.st->zero_phi;
  for (int q = tid; q < TX * TY * TZ; q += 256) {
    const int xx = q % TX, t = q / TX, yy = t % TY, zz = t / TY;
    const int x = x0 + xx, y = y0 + yy, z = z0 + zz;
    if (x >= nx || y >= ny || z >= nz) continue;
    const int id = z * plane + y * nx + x;
    const int rq = ((zz + 1) * RY + (yy + 1)) * RX + (xx + 1);
    T ev;
    if ((x + y + z) & 1) {
      const PlaneCoef<T> c = Cs[zz + 1];
      T acc = Rs[rq];
      acc = fma(c.cx, Rs[rq - 1] + Rs[rq + 1], acc);
      acc = fma(c.cy, Rs[rq - RX] + Rs[rq + RX], acc);
      acc = fma(c.czlo, Rs[rq - RX * RY], acc);
      acc = fma(c.czhi, Rs[rq + RX * RY], acc);
      ev = c.has_s ? acc / (c.diag + a.s[id]) : acc * c.invdiag;
    } else {
      ev = Rs[rq];
    }
    a.e_out[id] = ev;
    if (u.phi) apply_update(u, id, ev);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) restrict_kernel(MGArgs<T> a, LevelDesc F, LevelDesc C,
                                                       int skip_black) {
  pdl_enter();
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  if (I >= C.nx || J >= C.ny) return;
  restrict_cell(a, F, C, I, J, (int)blockIdx.z, skip_black);
}

// Direct FP64 form: the fine level's residual b - A phi after the pre-smoothing,
// restricted to the first coarse level (8-child mean, red children only when the
// black residuals vanish) and its squared norm summed on the way; the last block
// sums the per-block partials in a fixed order, takes the convergence decision
// (||r|| <= tol ||b||, ||b||^2 summed on the first check of a solve) and sets the
// loop condition.  phi after the pre-smoothing is the iterate the test accepts.
template <typename T>
__global__ void __launch_bounds__(256) restrict_check_kernel(MGArgs<T> fa, T* rc, LevelDesc F,
                                                             LevelDesc C, int skip_black,
                                                             CheckArgs ck) {
  pdl_enter();
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  double rr = 0.0, bb = 0.0, zz = 0.0;
  if (I < C.nx && J < C.ny)
    restrict_children<T, true>(fa, rc, nullptr, F, C, I, J, (int)blockIdx.z, skip_black, rr, bb,
                               ck.first);
  if (ck.first)
    block_sum3(rr, bb, zz);
  else
    block_sum1(rr);
  __shared__ bool last;
  const int nblk = gridDim.x * gridDim.y * gridDim.z;
  const int bid = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  if (tid == 0) {
    ck.partials[bid] = rr;
    ck.partials[nblk + bid] = ck.first ? bb : 0.0;
    __threadfence();
    const unsigned int prev = atomicAdd(&ck.stats->done_ctr, 1u);
    last = (prev == (unsigned)nblk - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double sr = 0.0, sb = 0.0;
  const volatile double* P = ck.partials;
  for (int q = tid; q < nblk; q += blockDim.x * blockDim.y) {
    sr += P[q];
    sb += P[nblk + q];
  }
  block_sum3(sr, sb, zz);
  if (tid == 0) {
    ck.stats->done_ctr = 0;
    const int cond = decide(ck.stats, sr, sb, 0.0, ck.first, ck.tol, ck.max_cycles,
                            ck.launches_per_cycle);
    if (ck.first) ck.stats->launches += ck.first_launches - 1;   // decide counted one
    if (ck.set_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)ck.cond_handle, cond);
  }
}

// Restriction with four threads per coarse cell (consecutive lanes): each sums
// the residuals of its children (positions q and q + 4 of the up to 2x2x2
// children, red only when the black residuals vanish), and two shuffles add the
// four partial sums ((s0 + s1) + (s2 + s3)).  The dependent chain per thread is
// one or two residuals instead of four to eight, for levels whose launch
// latency, not arithmetic, bounds the restriction.
template <typename T>
__global__ void __launch_bounds__(256) restrict4_kernel(MGArgs<T> a, LevelDesc F, LevelDesc C,
                                                        int skip_black) {
  pdl_enter();
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int q = (int)(t & 3);
  const long long cell = t >> 2;
  const bool own = cell < C.ncell;
  const int nxc = F.crx ? 2 : 1, nyc = F.cry ? 2 : 1, nzc = F.crz ? 2 : 1;
  const int nch = nxc * nyc * nzc;
  int I = 0, J = 0, K = 0;
  if (own) {
    const int rest = (int)(cell / C.nx);
    I = (int)(cell - (long long)rest * C.nx);
    K = rest / C.ny;
    J = rest - K * C.ny;
  }
  T sum = T(0), ssum = T(0);
  if (own) {
    for (int c = q; c < nch; c += 4) {
      const int di = c % nxc, dj = (c / nxc) % nyc, dk = c / (nxc * nyc);
      const int i = F.crx ? 2 * I + di : I, j = F.cry ? 2 * J + dj : J, k = F.crz ? 2 * K + dk : K;
      if (!(skip_black && ((i + j + k) & 1))) sum += cell_residual(a, F, i, j, k);
      if (a.s) ssum += a.s[lidx(F, i, j, k)];
    }
  }
  sum += __shfl_xor_sync(0xffffffffu, sum, 1);
  sum += __shfl_xor_sync(0xffffffffu, sum, 2);
  if (a.s) {
    ssum += __shfl_xor_sync(0xffffffffu, ssum, 1);
    ssum += __shfl_xor_sync(0xffffffffu, ssum, 2);
  }
  if (own && q == 0) {
    const T inv = T(1) / T(nch);
    const int idc = lidx(C, I, J, K);
    a.r[idc] = sum * inv;
    if (a.s) a.s[idc] = ssum * inv;
  }
}

// Prolongation + correction with one thread per fine cell (prolong_fine).
template <typename T>
__global__ void __launch_bounds__(256) prolong_fine_kernel(MGArgs<T> a, LevelDesc F, LevelDesc C,
                                                           int constant) {
  pdl_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= F.nx || j >= F.ny) return;
  prolong_fine(a, F, C, i, j, (int)blockIdx.z, constant);
}

template <typename T>
__global__ void __launch_bounds__(256) prolong_kernel(MGArgs<T> a, LevelDesc F, LevelDesc C,
                                                      int constant) {
  pdl_enter();
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  if (I >= C.nx || J >= C.ny) return;
  prolong_cell(a, F, C, I, J, (int)blockIdx.z, constant);
}

// Prolongation + correction onto the fine level in the FP64 form, tiled: the
// separable trilinear interpolation (3/4 own, 1/4 neighbour per direction) is
// done in y and then x once per coarse plane through shared memory, and then
// in z while the block marches up its coarse planes with the interpolated
// planes K-1, K, K+1 in registers.  An electrode beyond the coarse grid is a
// ghost plane holding -e (zero correction on the electrode face).  About 40
// FP64 operations per coarse cell against about 84 for the per-cell form
// (prolong_cell), which recomputes its neighbours' interpolations; used only
// where that arithmetic, not latency, bounds the launch.
// coarse columns (x, y) and planes per block; measured on the 256x256x32 stack
// (FP64, 500 steps): (32, 4, 4) 1227, (32, 8, 4) 1224, (32, 8, 2) 1216,
// (32, 4, 8) 1213, (32, 16, 4) 1207 Mcell-steps/s
constexpr int kPX = 32, kPY = 4, kPZ = 4;

template <typename T>
__global__ void __launch_bounds__(kPX* kPY) prolong_tiled_kernel(MGArgs<T> a, LevelDesc F,
                                                                LevelDesc C, T* fine) {
  pdl_enter();
  __shared__ T sE[kPY + 2][kPX + 2];     // coarse e of one plane: tile + periodic halo
  __shared__ T sY[2 * kPY][kPX + 2];     // interpolated in y: fine rows x coarse columns
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kPX + tx;
  const int I0 = blockIdx.x * kPX, J0 = blockIdx.y * kPY;
  const int I = I0 + tx, J = J0 + ty;
  const bool own = I < C.nx && J < C.ny;
  const int K0 = blockIdx.z * kPZ, K1 = min(C.nz, K0 + kPZ);
  T* e = a.e;
  T* ef = fine ? fine : e + F.off;       // the level's corrections, or phi (direct form)
  auto plane_xy = [&](int K, T out[4]) {
    __syncthreads();                     // the previous plane's readers are done with sE, sY
    for (int q = tid; q < (kPY + 2) * (kPX + 2); q += kPX * kPY) {
      const int r = q / (kPX + 2), col = q - r * (kPX + 2);
      int gy = (J0 - 1 + r) % C.ny, gx = (I0 - 1 + col) % C.nx;
      if (gy < 0) gy += C.ny;
      if (gx < 0) gx += C.nx;
      sE[r][col] = e[C.off + ((long long)K * C.ny + gy) * C.nx + gx];
    }
    __syncthreads();
    for (int q = tid; q < 2 * kPY * (kPX + 2); q += kPX * kPY) {
      const int fr = q / (kPX + 2), col = q - fr * (kPX + 2);
      const int ry = fr >> 1, b = fr & 1;
      sY[fr][col] = fma(T(0.75), sE[ry + 1][col], T(0.25) * sE[ry + 2 * b][col]);
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const T yc = sY[2 * ty + b][tx + 1];
      out[2 * b] = fma(T(0.75), yc, T(0.25) * sY[2 * ty + b][tx]);
      out[2 * b + 1] = fma(T(0.75), yc, T(0.25) * sY[2 * ty + b][tx + 2]);
    }
  };
  T xm[4], xc[4], xp[4];
  plane_xy(K0, xc);
  if (K0 > 0) {
    plane_xy(K0 - 1, xm);
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) xm[q] = -xc[q];
  }
  for (int K = K0; K < K1; ++K) {
    if (K + 1 < C.nz) {
      plane_xy(K + 1, xp);
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) xp[q] = -xc[q];
    }
    if (own) {
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        T* lo = ef + ((long long)(2 * K) * F.ny + 2 * J + b) * F.nx + 2 * I;
        T* hi = lo + (long long)F.ny * F.nx;
        lo[0] += fma(T(0.75), xc[2 * b], T(0.25) * xm[2 * b]);
        lo[1] += fma(T(0.75), xc[2 * b + 1], T(0.25) * xm[2 * b + 1]);
        hi[0] += fma(T(0.75), xc[2 * b], T(0.25) * xp[2 * b]);
        hi[1] += fma(T(0.75), xc[2 * b + 1], T(0.25) * xp[2 * b + 1]);
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) { xm[q] = xc[q]; xc[q] = xp[q]; }
  }
}

template <typename T>
__global__ void __launch_bounds__(kTailThreads) tail_kernel(MGArgs<T> g, TailArgs t) {
  extern __shared__ __align__(16) unsigned char tail_smem[];
  pdl_enter();
  tail_vcycle<T>(g, t, tail_smem);
}

// grid (x chunk, row chunk, z chunk): block z owns planes [z kchunk, (z+1) kchunk)
template <typename T, bool SC>
__global__ void __launch_bounds__(kResidBX* kResidBY) resid_kernel(ResidArgs a) {
  pdl_enter();
  const int i = blockIdx.x * kResidBX + threadIdx.x;
  const int j = blockIdx.y * kResidBY + threadIdx.y;
  const int k0 = blockIdx.z * a.kchunk;
  const int k1 = min(a.nz, k0 + a.kchunk);
  double acc_r = 0.0, acc_b = 0.0, acc_rho = 0.0;
  if (i < a.nx && j < a.ny) resid_column<T, SC>(a, i, j, k0, k1, acc_r, acc_b, acc_rho);
  if (a.no_stats) return;
  // ||b||^2 is summed on the first residual of a solve only, ||rho||^2 with carriers only
  if (SC || a.first)
    block_sum3(acc_r, acc_b, acc_rho);
  else
    block_sum1(acc_r);
  __shared__ bool last;
  const int nblk = gridDim.x * gridDim.y * gridDim.z;
  const int bid = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  if (tid == 0) {
    a.partials[bid] = acc_r;
    a.partials[nblk + bid] = acc_b;
    a.partials[2 * nblk + bid] = acc_rho;
    __threadfence();
    const unsigned int prev = atomicAdd(&a.stats->done_ctr, 1u);
    last = (prev == (unsigned)nblk - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // fixed-order sum of the partials (deterministic)
  double sr = 0.0, sb = 0.0, sq = 0.0;
  const volatile double* P = a.partials;
  for (int q = tid; q < nblk; q += blockDim.x * blockDim.y) {
    sr += P[q];
    sb += P[nblk + q];
    sq += P[2 * nblk + q];
  }
  block_sum3(sr, sb, sq);
  if (tid == 0) {
    a.stats->done_ctr = 0;
    if (a.norm_out) {
      *a.norm_out = sqrt(sr);
      return;
    }
    if (a.reject_ref) {
      // keep a learned correction only if it lowered ||r|| or already meets the
      // test; a rejected one leaves the statistics to the residual of the restored
      // guess (the IF body), which also sets the loop condition
      const double rn = sqrt(sr), scale = fmax(sqrt(sb), sqrt(sq));
      const bool met = rn <= a.tol * scale;
      const int reject = !isfinite(rn) || !isfinite(scale) || (!(rn < *a.reject_ref) && !met);
      cudaGraphSetConditional((cudaGraphConditionalHandle)a.reject_handle, reject);
      if (reject) {
        a.stats->nn_rejected += 1;
        a.stats->launches += 1;
        return;
      }
    }
    const int cond = decide(a.stats, sr, sb, sq, a.first, a.tol, a.max_cycles, a.launches_per_cycle,
                            a.adapt_max, a.launches_per_vcycle, a.inner_fixed);
    if (a.set_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)a.cond_handle, cond);
  }
}

// e = A^-1 r on one level by its dense inverse (row-major, n x n): one warp per
// row, lanes over columns, a fixed-order shuffle reduction.  Used for a level
// that replaces the single-CTA tail in the FP64 form: the matrix-vector product
// spreads over the SMs where the tail's V-cycle would run on one.
template <typename T>
__global__ void __launch_bounds__(256) dense_solve_kernel(const T* __restrict__ inv, int n,
                                                          const T* __restrict__ r,
                                                          T* __restrict__ e) {
  pdl_enter();
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const T* a = inv + (size_t)row * n;
  T acc = T(0);
  for (int c = lane; c < n; c += 32) acc = fma(__ldg(a + c), r[c], acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) e[row] = acc;
}

template <typename T>
__global__ void __launch_bounds__(256) update_kernel(double* __restrict__ phi, const T* __restrict__ e0,
                                                     long long n, const DevStats* stats,
                                                     double clamp, T* zero_e) {
  pdl_enter();
  const Upd u{phi, clamp, stats->zero_phi};
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    apply_update(u, t, e0[t]);
    if (zero_e) zero_e[t] = T(0);   // the next outer iteration starts from a zero correction
  }
}

__global__ void inner_arm_kernel(const DevStats* st, unsigned long long handle) {
  pdl_enter();
  cudaGraphSetConditional((cudaGraphConditionalHandle)handle, st->inner_left > 0 ? 1 : 0);
}

__global__ void inner_countdown_kernel(DevStats* st, unsigned long long handle) {
  pdl_enter();
  const int left = st->inner_left - 1;
  st->inner_left = left;
  cudaGraphSetConditional((cudaGraphConditionalHandle)handle, left > 0 ? 1 : 0);
}

// threads per block: 256, halved to 128 when the grid would hold fewer than two
// blocks per SM, so small levels spread over more SMs (their FP64 arithmetic,
// at 2 DFMA per clock per SM, bounds them)
int spread_threads(long long items) {
  int t = 256;
  while (t > 128 && items < 2LL * 152 * t) t >>= 1;
  return t;
}

// 2-D block over (x items, rows): x extent a power of two up to 128
void block_shape(int nxi, int ny, dim3& block, dim3& grid, int nz, int threads = 256) {
  int bx = 1;
  while (bx < nxi && bx < 128 && bx < threads) bx <<= 1;
  int by = threads / bx;
  if (by > ny) { by = 1; while (by < ny) by <<= 1; }
  block = dim3(bx, by, 1);
  grid = dim3((nxi + bx - 1) / bx, (ny + by - 1) / by, nz);
}

}  // namespace

template <typename T>
void launch_smooth(const MGArgs<T>& a, const LevelDesc& L, int color, int zero_init,
                   const UpdateArgs* upd, cudaStream_t s, const DevStats* zero_stats) {
  if (!zero_init && !upd) {
    // plain sweeps: two planes per thread on large FP32 levels (more loads in
    // flight for an issue-bound sweep), one elsewhere (FP64 arithmetic bounds it)
    const int kz = (sizeof(T) == sizeof(float) && L.ncell >= (1LL << 20)) ? 2 : 1;
    dim3 block, grid;
    block_shape((L.nx + 1) >> 1, L.ny, block, grid, (L.nz + kz - 1) / kz,
                spread_threads((long long)((L.nx + 1) >> 1) * L.ny * ((L.nz + kz - 1) / kz)));
    if (kz == 2)
      launch_k(smooth_kz_kernel<T, 2>, grid, block, 0, s, a, L, color, zero_stats);
    else
      launch_k(smooth_kz_kernel<T, 1>, grid, block, 0, s, a, L, color, zero_stats);
    return;
  }
  dim3 block, grid;
  block_shape((L.nx + 1) >> 1, L.ny, block, grid, L.nz,
              spread_threads((long long)((L.nx + 1) >> 1) * L.ny * L.nz));
  Upd u{nullptr, 0.0, 0};
  const DevStats* st = nullptr;
  if (upd) { u.phi = upd->phi; u.clamp = upd->clamp; st = upd->stats; }
  launch_k(smooth_kernel<T>, grid, block, 0, s, a, L, color, zero_init, u, st, zero_stats);
}

namespace {
template <typename T, int TX, int TY, int TZ>
size_t rb_smem_bytes(int zero_init) {
  constexpr int RZ = TZ + 2;
  const size_t head = ((RZ * sizeof(PlaneCoef<T>) + 15) / 16) * 16;
  const size_t en = zero_init ? 0 : (size_t)(TX + 4) * (TY + 4) * (TZ + 4);
  return head + (en + (size_t)(TX + 2) * (TY + 2) * RZ) * sizeof(T);
}

template <typename T, int TX, int TY, int TZ>
void launch_rb(const RBArgs<T>& a, cudaStream_t s) {
  const size_t smem = rb_smem_bytes<T, TX, TY, TZ>(a.zero_init);
  const dim3 grid((a.nx + TX - 1) / TX, (a.ny + TY - 1) / TY, (a.nz + TZ - 1) / TZ);
  launch_k(smooth_rb_kernel<T, TX, TY, TZ>, grid, dim3(256), smem, s, a);
}

template <typename T, int TX, int TY, int TZ>
cudaError_t rb_prepare_one() {
  return cudaFuncSetAttribute(smooth_rb_kernel<T, TX, TY, TZ>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)rb_smem_bytes<T, TX, TY, TZ>(0));
}
}  // namespace

// shared-memory opt-in of the fused sweep kernels on the current device
template <typename T>
cudaError_t smooth_rb_prepare() {
  cudaError_t e = rb_prepare_one<T, 32, 16, 8>();
  return e != cudaSuccess ? e : rb_prepare_one<T, 16, 8, 4>();
}

// tile of the fused sweep for a level: the large tile where it still gives
// enough blocks, a small one otherwise (0: not eligible)
template <typename T>
int smooth_rb_tile(const LevelDesc& L) {
  if (sizeof(T) != sizeof(float)) return 0;
  if ((L.nx & 1) || (L.ny & 1)) return 0;
  if (L.nx >= 32 && L.ny >= 16 && L.ncell >= (1LL << 20)) return 2;   // 32 x 16 x 8
  if (L.nx >= 16 && L.ny >= 8 && L.ncell >= (1LL << 14)) return 1;    // 16 x 8 x 4
  return 0;
}

template <typename T>
void launch_smooth_rb(const MGArgs<T>& a, const LevelDesc& L, const T* e_in, T* e_out,
                      int zero_init, const UpdateArgs* upd, cudaStream_t s) {
  RBArgs<T> r{};
  r.e_in = e_in;
  r.e_out = e_out;
  r.r = a.r + L.off;
  r.s = a.s ? a.s + L.off : nullptr;
  r.coef = a.coef + L.coef_off;
  r.nx = L.nx; r.ny = L.ny; r.nz = L.nz;
  r.zero_init = zero_init;
  r.u = Upd{nullptr, 0.0, 0};
  if (upd) { r.u.phi = upd->phi; r.u.clamp = upd->clamp; r.st = upd->stats; }
  if (smooth_rb_tile<T>(L) == 2)
    launch_rb<T, 32, 16, 8>(r, s);
  else
    launch_rb<T, 16, 8, 4>(r, s);
}

dim3 check_grid(const LevelDesc& C) {
  dim3 block, grid;
  block_shape(C.nx, C.ny, block, grid, C.nz);
  return grid;
}

void launch_restrict_check(const MGArgs<double>& fa, double* rc, const LevelDesc& F,
                           const LevelDesc& C, int nu1, const CheckArgs& ck, cudaStream_t s) {
  dim3 block, grid;
  block_shape(C.nx, C.ny, block, grid, C.nz);
  launch_k(restrict_check_kernel<double>, grid, block, 0, s, fa, rc, F, C,
           black_residual_zero(F, nu1), ck);
}

// Latency-bound FP32 levels: the per-thread chains of the one-thread-per-coarse-
// cell transfers dominate up to this size.  Measured on 256x256x32, 500 steps
// (Mcell-steps/s, mixed / fast form): none 1781 / 2735, up to 4096 cells
// 1799 / 2761, up to 32768 cells 1804 / 2775; larger FP32 levels lose.  FP64
// levels use the split kernels at every size (+2.2% FP64).
constexpr long long kSmallTransfer = 32768;

template <typename T>
void launch_restrict(const MGArgs<T>& a, const LevelDesc& F, const LevelDesc& C, int nu1,
                     cudaStream_t s) {
  if (sizeof(T) == sizeof(double) || C.ncell <= kSmallTransfer) {
    // four threads per coarse cell where latency bounds the restriction: FP64
    // levels, and FP32 levels up to kSmallTransfer coarse cells
    const long long threads = 4 * C.ncell;
    launch_k(restrict4_kernel<T>, dim3((unsigned)((threads + 255) / 256)), dim3(256), 0, s, a, F, C,
             black_residual_zero(F, nu1));
    return;
  }
  dim3 block, grid;
  block_shape(C.nx, C.ny, block, grid, C.nz, spread_threads(C.ncell));
  launch_k(restrict_kernel<T>, grid, block, 0, s, a, F, C, black_residual_zero(F, nu1));
}

template <typename T>
void launch_prolong(const MGArgs<T>& a, const LevelDesc& F, const LevelDesc& C, int constant,
                    cudaStream_t s, bool tiled, T* fine) {
  if (fine || (tiled && F.crx && F.cry && F.crz && !constant)) {
    const dim3 grid((C.nx + kPX - 1) / kPX, (C.ny + kPY - 1) / kPY, (C.nz + kPZ - 1) / kPZ);
    launch_k(prolong_tiled_kernel<T>, grid, dim3(kPX, kPY), 0, s, a, F, C, fine);
    return;
  }
  if (sizeof(T) == sizeof(double) || F.ncell <= kSmallTransfer) {
    // one thread per fine cell, a 15-operation chain instead of 84 per coarse
    // cell, where latency bounds the prolongation: FP64 levels, and FP32 levels
    // up to kSmallTransfer fine cells
    dim3 block, grid;
    block_shape(F.nx, F.ny, block, grid, F.nz, spread_threads(F.ncell));
    launch_k(prolong_fine_kernel<T>, grid, block, 0, s, a, F, C, constant);
    return;
  }
  dim3 block, grid;
  block_shape(C.nx, C.ny, block, grid, C.nz, spread_threads(C.ncell));
  launch_k(prolong_kernel<T>, grid, block, 0, s, a, F, C, constant);
}

template <typename T>
void launch_dense_solve(const T* inv, int n, const T* r, T* e, cudaStream_t s) {
  launch_k(dense_solve_kernel<T>, dim3((unsigned)((n + 7) / 8)), dim3(256), 0, s, inv, n, r, e);
}

template <typename T>
size_t tail_smem_bytes(long long elems, bool has_s) {
  return (size_t)elems * sizeof(T) * (has_s ? 3 : 2);
}

template <typename T>
cudaError_t tail_prepare(size_t smem) {
  return cudaFuncSetAttribute(tail_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <typename T>
void launch_tail(const MGArgs<T>& a, const TailArgs& t, size_t smem, cudaStream_t s) {
  launch_k(tail_kernel<T>, dim3(1), dim3(kTailThreads), smem, s, a, t);
}

template <typename T>
void launch_resid(const ResidArgs& a, cudaStream_t s) {
  dim3 block(kResidBX, kResidBY);
  dim3 grid((a.nx + kResidBX - 1) / kResidBX, (a.ny + kResidBY - 1) / kResidBY,
            (a.nz + a.kchunk - 1) / a.kchunk);
  if (a.s_out)
    launch_k(resid_kernel<T, true>, grid, block, 0, s, a);
  else
    launch_k(resid_kernel<T, false>, grid, block, 0, s, a);
}

template <typename T>
void launch_update(double* phi, const T* e0, long long n, const DevStats* stats, double clamp,
                   cudaStream_t s, T* zero_e) {
  long long b = (n + 255) / 256;
  if (b > 152LL * 16) b = 152LL * 16;
  launch_k(update_kernel<T>, dim3((int)b), dim3(256), 0, s, phi, e0, n, stats, clamp, zero_e);
}

void launch_inner_arm(const DevStats* st, unsigned long long handle, cudaStream_t s) {
  launch_k(inner_arm_kernel, dim3(1), dim3(1), 0, s, st, handle);
}

void launch_inner_countdown(DevStats* st, unsigned long long handle, cudaStream_t s) {
  launch_k(inner_countdown_kernel, dim3(1), dim3(1), 0, s, st, handle);
}

// e^{+u}, e^{-u} of n arguments with the carrier routine of the residual kernel
// (grid-stride; exposed so its error can be checked on its own)
__global__ void __launch_bounds__(256) carrier_exp_kernel(const double* __restrict__ u,
                                                          double* __restrict__ ep,
                                                          double* __restrict__ em, long long n) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) {
    double a, b;
    exp_pm(u[i], a, b);
    ep[i] = a;
    em[i] = b;
  }
}

cudaError_t launch_carrier_exp(const double* u, double* ep, double* em, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  long long b = (n + 255) / 256;
  if (b > 152LL * 8) b = 152LL * 8;
  carrier_exp_kernel<<<(int)b, 256, 0, s>>>(u, ep, em, n);
  return cudaGetLastError();
}

#define FX_INST(T)                                                                              \
  template void launch_smooth<T>(const MGArgs<T>&, const LevelDesc&, int, int,                  \
                                 const UpdateArgs*, cudaStream_t, const DevStats*);             \
  template int smooth_rb_tile<T>(const LevelDesc&);                                             \
  template cudaError_t smooth_rb_prepare<T>();                                                  \
  template void launch_smooth_rb<T>(const MGArgs<T>&, const LevelDesc&, const T*, T*, int,      \
                                    const UpdateArgs*, cudaStream_t);                           \
  template void launch_restrict<T>(const MGArgs<T>&, const LevelDesc&, const LevelDesc&, int,   \
                                   cudaStream_t);                                               \
  template void launch_prolong<T>(const MGArgs<T>&, const LevelDesc&, const LevelDesc&, int,    \
                                  cudaStream_t, bool, T*);                                      \
  template size_t tail_smem_bytes<T>(long long, bool);                                          \
  template cudaError_t tail_prepare<T>(size_t);                                                 \
  template void launch_tail<T>(const MGArgs<T>&, const TailArgs&, size_t, cudaStream_t);        \
  template void launch_dense_solve<T>(const T*, int, const T*, T*, cudaStream_t);               \
  template void launch_resid<T>(const ResidArgs&, cudaStream_t);                                \
  template void launch_update<T>(double*, const T*, long long, const DevStats*, double,         \
                                 cudaStream_t, T*);
FX_INST(double)
FX_INST(float)
#undef FX_INST

}  // namespace fx

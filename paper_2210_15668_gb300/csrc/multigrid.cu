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

#include <algorithm>

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
//
// SCALED (the direct FP64 form's fine level): r holds b / diag and the
// coefficients are divided by the diagonal on the host, so a cell is six FP64
// operations (two additions, four multiply-adds) instead of seven.
template <typename T, int KZ, bool SCALED = false>
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
    if constexpr (SCALED) a.e[id] = acc;
    else if (!c[q].has_s) a.e[id] = acc * c[q].invdiag;
    else a.e[id] = a.sinv ? acc * a.sinv[id - L.off] : acc / (c[q].diag + a.s[id]);
  }
}

// bs = b / diag on every cell of the fine level (once per solve of the direct form)
__global__ void __launch_bounds__(256) scale_rhs_kernel(const double* __restrict__ b,
                                                        const PlaneCoef<double>* __restrict__ coef,
                                                        long long plane, long long n,
                                                        double* __restrict__ bs) {
  pdl_enter();
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    bs[t] = b[t] * __ldg(&coef[t / plane].invdiag);
}

// ---- fused red-black sweep (one launch per full sweep, out of place) -------------------
// One red-black Gauss-Seidel sweep of a level (red cells, then black cells) in
// one launch, reading e_in and writing e_out.  A block owns a 32 x 16 lateral
// tile and marches up a chunk of planes.  Each plane of e_in (with a two-cell
// lateral halo) and of r (one-cell halo) is copied into a shared-memory ring a
// few planes ahead of its use (cp.async).  At each step the block relaxes the
// red cells of one plane, tile plus one-cell halo (the halo's red values are
// recomputed from the same inputs and operations as in the block that owns those
// cells, so they are identical), then the black cells of the plane below against
// the new red values of its three planes, and writes both colours of that plane.
// Red cells are (i + j + k) even, as in the colour sweeps.  Every cell sees the
// operations of smooth_pair in the same order, so one launch equals the red
// sweep followed by the black sweep bit for bit, while each array element is read
// from memory and written once per full sweep instead of once per colour.
// Lateral sizes must be even and at least the tile's (one periodic wrap covers
// the halo); planes beyond the level are the zero of the correction equation's
// Dirichlet faces.  With zero_init the sweep starts from e = 0 (e_in unused).
// With u.phi set, phi += e of both colours (clamped) follows.
template <typename T>
struct RBArgs {
  const T* e_in;            // level-relative
  T* e_out;                 // level-relative
  const T* r;               // level-relative
  const T* s;               // level-relative Newton shift (null without SC)
  const T* sinv;            // level-relative 1 / (diag + s): multiply instead of divide
  const PlaneCoef<T>* coef; // the level's planes
  int nx, ny, nz;
  int kz;                   // planes per block (z chunk)
  int zero_init;
  Upd u;
  const DevStats* st;       // zero_phi flag for the fused update
};

// asynchronous 16-byte global -> shared copy (zero-filled when !valid)
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src),
               "r"(valid ? 16 : 0)
               : "memory");
}

__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Shared-memory planes are 40 floats wide: global x0 - 4 .. x0 + 35 (local lx =
// x - x0 + 4), staged as ten 16-byte chunks per row.  The e planes hold rows
// y0 - 2 .. y0 + 17 (two-cell halo), the r (s) planes rows y0 - 1 .. y0 + 16.
constexpr int kRbTX = 32, kRbTY = 16;          // lateral tile, 256 threads
constexpr int kRbD = 1;                        // planes staged ahead of use
constexpr int kRbW = 40, kRbCH = 10;           // row width (floats) and 16-byte chunks per row
constexpr int kRbEY = kRbTY + 4, kRbEP = kRbEY * kRbW;
constexpr int kRbRY = kRbTY + 2, kRbRP = kRbRY * kRbW;
constexpr int kRbNE = kRbD + 3, kRbNR = kRbD + 5;   // ring slots (see the step loop)
constexpr int kRbKZ = 128;                          // planes per block at most
constexpr long long kRbMinCells = 1LL << 23;        // smaller levels keep the colour sweeps
constexpr int kRbCoefBytes = (kRbKZ + 2) * (int)sizeof(PlaneCoef<float>);

__global__ void __launch_bounds__(256) smooth_rb_kernel(RBArgs<float> a) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PlaneCoef<float>* Cs = reinterpret_cast<PlaneCoef<float>*>(smem_raw);   // planes z0-1 .. z1
  float* Es = reinterpret_cast<float*>(smem_raw + kRbCoefBytes);  // kRbNE e planes (not with zero_init)
  float* Rs = Es + (a.zero_init ? 0 : kRbNE * kRbEP);        // kRbNR planes: r, then new red values
  float* Ss = Rs + kRbNR * kRbRP;                            // kRbNR planes of s (semiconductor)
  const int t = threadIdx.x;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int plane = nx * ny;
  const int x0 = blockIdx.x * kRbTX, y0 = blockIdx.y * kRbTY;
  const int z0 = blockIdx.z * a.kz, z1 = min(z0 + a.kz, nz);
  auto wrapx = [&](int x) { return x < 0 ? x + nx : (x >= nx ? x - nx : x); };
  auto wrapy = [&](int y) { return y < 0 ? y + ny : (y >= ny ? y - ny : y); };
  // staging items of this thread (fixed across planes): e chunk t (< 200), r/s chunk t (< 180)
  const bool has_e = !a.zero_init && t < kRbEY * kRbCH;
  const bool has_r = t < kRbRY * kRbCH;
  const int ch = t % kRbCH;
  const int e_soff = (t / kRbCH) * kRbW + ch * 4;
  const int e_goff = wrapy(y0 - 2 + t / kRbCH) * nx + wrapx(x0 - 4 + ch * 4);
  const int r_soff = e_soff;                                   // same row/chunk layout
  const int r_goff = wrapy(y0 - 1 + t / kRbCH) * nx + wrapx(x0 - 4 + ch * 4);
  const int nunits = z1 - z0 + 4;                               // e planes z0-2 .. z1+1
  auto stage = [&](int j) {
    if (j < nunits) {
      const int z = z0 - 2 + j;
      const bool zin = z >= 0 && z < nz;
      const int zoff = zin ? z * plane : 0;
      if (has_e) cp_async16(Es + (j % kRbNE) * kRbEP + e_soff, a.e_in + zoff + e_goff, zin);
      if (has_r && z >= z0 - 1 && z <= z1) {
        cp_async16(Rs + (j % kRbNR) * kRbRP + r_soff, a.r + zoff + r_goff, zin);
        if (a.sinv) cp_async16(Ss + (j % kRbNR) * kRbRP + r_soff, a.sinv + zoff + r_goff, zin);
        else if (a.s) cp_async16(Ss + (j % kRbNR) * kRbRP + r_soff, a.s + zoff + r_goff, zin);
      }
    }
    cp_async_commit();   // one group per unit, empty past the end
  };
  // red items of this thread: item t and t + 256 of the 18 rows x 17 red cells of the
  // r region (x0 - 1 .. x0 + 32); black item: row t / 16, pair t % 16 of the tile
  const int it0 = t, it1 = t + 256;
  const int ry0 = it0 / 17, rk0 = it0 % 17;
  const int ry1 = it1 / 17, rk1 = it1 % 17;
  const bool red1 = it1 < kRbRY * 17;
  const int by = t >> 4, bk = t & 15;
  const int gy_b = y0 + by;
  const bool bout = (x0 + 2 * bk) < nx && gy_b < ny;
  Upd u = a.u;
  if (u.phi) u.zero = a.st->zero_phi;

  for (int j = 0; j < kRbD + 2; ++j) stage(j);
  // coefficients of every plane the block relaxes (the first barrier publishes them)
  for (int q = t; q < z1 - z0 + 2; q += 256) {
    const int z = z0 - 1 + q;
    if (z >= 0 && z < nz) Cs[q] = ldg_struct(a.coef + z);
  }
  // step i: red cells of plane p = z0 - 1 + i (units i .. i + 2 staged), then the
  // black cells of plane p - 1 and both colours of it written out
  int se = 0, sr = 0;   // ring slot of unit i in the e and r rings
  for (int i = 0; i < z1 - z0 + 2; ++i) {
    stage(i + kRbD + 2);
    cp_async_wait<kRbD>();
    __syncthreads();
    const int p = z0 - 1 + i;
    const int se1 = se + 1 == kRbNE ? 0 : se + 1, se2 = se1 + 1 == kRbNE ? 0 : se1 + 1;
    const int sr1 = sr + 1 == kRbNR ? 0 : sr + 1, srm = sr == 0 ? kRbNR - 1 : sr - 1;
    if (p >= 0 && p < nz) {
      const PlaneCoef<float> c = Cs[i];
      float* R = Rs + sr1 * kRbRP;
      const float* S = Ss + sr1 * kRbRP;
      const float* Ec = Es + se1 * kRbEP;   // plane p
      const float* Ed = Es + se * kRbEP;    // plane p - 1
      const float* Eu = Es + se2 * kRbEP;   // plane p + 1
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (h == 1 && !red1) break;
        const int ry = h ? ry1 : ry0, k = h ? rk1 : rk0;
        // red cells of the row: local lx = 3 or 4, then every second one
        const int lx = 3 + ((3 + y0 - 1 + ry + p) & 1) + 2 * k;
        const int q = ry * kRbW + lx;
        float ev;
        if (a.zero_init) {
          const float d = c.has_s ? (a.sinv ? S[q] : 1.0f / (c.diag + S[q])) : c.invdiag;
          ev = R[q] * d;
        } else {
          const int e = q + kRbW;             // the e planes start one row lower
          float acc = R[q];
          acc = fmaf(c.cx, Ec[e - 1] + Ec[e + 1], acc);
          acc = fmaf(c.cy, Ec[e - kRbW] + Ec[e + kRbW], acc);
          acc = fmaf(c.czlo, Ed[e], acc);
          acc = fmaf(c.czhi, Eu[e], acc);
          ev = c.has_s ? (a.sinv ? acc * S[q] : acc / (c.diag + S[q])) : acc * c.invdiag;
        }
        R[q] = ev;
      }
    }
    __syncthreads();
    const int pb = p - 1;
    if (pb >= z0 && pb < z1 && bout) {
      const PlaneCoef<float> c = Cs[i - 1];
      const float* Rc = Rs + sr * kRbRP;    // plane pb
      const float* Rd = Rs + srm * kRbRP;   // plane pb - 1
      const float* Ru = Rs + sr1 * kRbRP;   // plane pb + 1 (red values of this step)
      const float* S = Ss + sr * kRbRP;
      // the pair (x0 + 2 bk, x0 + 2 bk + 1): its black cell is the second when x0 + 2 bk is red
      const int second = ((gy_b + pb) & 1) == 0;
      const int q0 = (by + 1) * kRbW + 4 + 2 * bk;
      const int qb = q0 + second;
      float acc = Rc[qb];
      acc = fmaf(c.cx, Rc[qb - 1] + Rc[qb + 1], acc);
      acc = fmaf(c.cy, Rc[qb - kRbW] + Rc[qb + kRbW], acc);
      acc = fmaf(c.czlo, Rd[qb], acc);
      acc = fmaf(c.czhi, Ru[qb], acc);
      const float eb = c.has_s ? (a.sinv ? acc * S[qb] : acc / (c.diag + S[qb])) : acc * c.invdiag;
      const float er = Rc[q0 + 1 - second];
      const int id = pb * plane + gy_b * nx + x0 + 2 * bk;
      const float2 v = second ? make_float2(er, eb) : make_float2(eb, er);
      *reinterpret_cast<float2*>(a.e_out + id) = v;
      if (u.phi) {
        apply_update(u, id, v.x);
        apply_update(u, id + 1, v.y);
      }
    }
    se = se1;
    sr = sr1;
  }
  cp_async_wait<0>();
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
  float rr = 0.0f, bb = 0.0f;   // FP32 sums of the squares (see restrict_children)
  if (I < C.nx && J < C.ny)
    restrict_children<T, true, float>(fa, rc, nullptr, F, C, I, J, (int)blockIdx.z, skip_black, rr,
                                      bb, ck.first);
  block_sum2f(rr, bb);
  double zz = 0.0;
  __shared__ bool last;
  const int nblk = gridDim.x * gridDim.y * gridDim.z;
  const int bid = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  if (tid == 0) {
    ck.partials[bid] = (double)rr;
    ck.partials[nblk + bid] = ck.first ? (double)bb : 0.0;
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
template <typename T, int SC, bool DF = false>
__global__ void __launch_bounds__(kResidBX* kResidBY) resid_kernel(ResidArgs a) {
  pdl_enter();
  const int i = blockIdx.x * kResidBX + threadIdx.x;
  const int j = blockIdx.y * kResidBY + threadIdx.y;
  const int k0 = blockIdx.z * a.kchunk;
  const int k1 = min(a.nz, k0 + a.kchunk);
  double acc_r = 0.0, acc_b = 0.0, acc_rho = 0.0;
  if constexpr (DF) {
    float fr = 0.0f, fb = 0.0f;
    if (i < a.nx && j < a.ny) resid_column_df<T, SC>(a, i, j, k0, k1, fr, fb, acc_rho);
    if (a.no_stats) return;
    // the squared norms within the block in FP32 (no FP64 work per cell), across
    // blocks in FP64 below; ||rho||^2 in FP64
    block_sum2f(fr, fb);
    if (SC) block_sum1(acc_rho);
    acc_r = (double)fr;
    acc_b = (double)fb;
  } else {
    if (i < a.nx && j < a.ny) resid_column<T, SC>(a, i, j, k0, k1, acc_r, acc_b, acc_rho);
    if (a.no_stats) return;
    // ||b||^2 is summed on the first residual of a solve only, ||rho||^2 with carriers only
    if (SC || a.first)
      block_sum3(acc_r, acc_b, acc_rho);
    else
      block_sum1(acc_r);
  }
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
  const Upd u{phi, clamp, stats->zero_phi, (float)clamp};
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
  Upd u{nullptr, 0.0, 0, 0.0f};
  const DevStats* st = nullptr;
  if (upd) { u.phi = upd->phi; u.clamp = upd->clamp; u.clampf = (float)upd->clamp; st = upd->stats; }
  launch_k(smooth_kernel<T>, grid, block, 0, s, a, L, color, zero_init, u, st, zero_stats);
}

namespace {
size_t rb_smem_bytes(int zero_init, bool has_s) {
  return kRbCoefBytes +
         ((zero_init ? 0 : (size_t)kRbNE * kRbEP) + (size_t)kRbNR * kRbRP * (has_s ? 2 : 1)) *
             sizeof(float);
}

// planes per block: the largest power of two (4 .. kRbKZ) that still gives six
// blocks per SM
int rb_kz(const LevelDesc& L) {
  const long long tiles = (long long)((L.nx + kRbTX - 1) / kRbTX) * ((L.ny + kRbTY - 1) / kRbTY);
  int kz = 1;
  while (kz < L.nz && kz < kRbKZ) kz <<= 1;
  while (kz > 4 && tiles * ((L.nz + kz - 1) / kz) < 6LL * 152) kz >>= 1;
  return kz;
}
}  // namespace

// shared-memory opt-in of the fused sweep kernel on the current device
template <typename T>
cudaError_t smooth_rb_prepare() {
  return cudaFuncSetAttribute(smooth_rb_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)rb_smem_bytes(0, true));
}

// 1 where the level takes the fused sweep, 0 where it keeps the colour sweeps.
// FP32 levels whose lateral sizes are multiples of 4 and at least 36 x 16 (one
// periodic wrap covers the staged window; the 16-byte chunks never straddle it)
// and that hold at least kRbMinCells cells.  Measured on GB300 inside the CUDA
// graph of a step: on DRAM-bound levels (512 x 512 x 128) the fused sweep wins
// (mixed Newton form 2110 -> 2264 Mcell-steps/s); on L2-resident levels of
// 2-4 M cells the colour sweeps overlap better under programmatic launch and
// win (256 x 256 x 32: 1578 vs 1494; 256 x 256 x 64: 1749 vs 1635).
template <typename T>
int smooth_rb_tile(const LevelDesc& L, bool) {
  if (sizeof(T) != sizeof(float)) return 0;
  if ((L.nx & 3) || (L.ny & 1) || L.nx < 36 || L.ny < kRbTY || L.ncell < kRbMinCells) return 0;
  return 1;
}

// colour sweep of the direct FP64 form's fine level on b / diag with scaled coefficients
void launch_smooth_scaled(const MGArgs<double>& a, const LevelDesc& L, int color, cudaStream_t s,
                          const DevStats* zero_stats) {
  dim3 block, grid;
  block_shape((L.nx + 1) >> 1, L.ny, block, grid, L.nz,
              spread_threads((long long)((L.nx + 1) >> 1) * L.ny * L.nz));
  launch_k(smooth_kz_kernel<double, 1, true>, grid, block, 0, s, a, L, color, zero_stats);
}

void launch_scale_rhs(const double* b, const PlaneCoef<double>* coef, int nx, int ny, int nz, double* bs,
                      cudaStream_t s) {
  const long long plane = (long long)nx * ny, n = plane * nz;
  long long blocks = (n + 255) / 256;
  if (blocks > 152LL * 8) blocks = 152LL * 8;
  launch_k(scale_rhs_kernel, dim3((unsigned)blocks), dim3(256), 0, s, b, coef, plane, n, bs);
}

template <typename T>
void launch_smooth_rb(const MGArgs<T>& a, const LevelDesc& L, const T* e_in, T* e_out,
                      int zero_init, const UpdateArgs* upd, cudaStream_t s) {
  if constexpr (sizeof(T) == sizeof(float)) {
    RBArgs<float> r{};
    r.e_in = e_in;
    r.e_out = e_out;
    r.r = a.r + L.off;
    r.s = a.s ? a.s + L.off : nullptr;
    r.sinv = a.sinv;
    r.coef = a.coef + L.coef_off;
    r.nx = L.nx; r.ny = L.ny; r.nz = L.nz;
    r.kz = rb_kz(L);
    r.zero_init = zero_init;
    r.u = Upd{nullptr, 0.0, 0, 0.0f};
    if (upd) { r.u.phi = upd->phi; r.u.clamp = upd->clamp; r.u.clampf = (float)upd->clamp; r.st = upd->stats; }
    const dim3 grid((L.nx + kRbTX - 1) / kRbTX, (L.ny + kRbTY - 1) / kRbTY,
                    (L.nz + r.kz - 1) / r.kz);
    launch_k(smooth_rb_kernel, grid, dim3(256), rb_smem_bytes(zero_init, r.s != nullptr), s, r);
  }
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
void launch_resid(const ResidArgs& a_in, cudaStream_t s) {
  ResidArgs a = a_in;
  a.warp_rows = a.nx % 32 == 0;
  dim3 block(kResidBX, kResidBY);
  dim3 grid((a.nx + kResidBX - 1) / kResidBX, (a.ny + kResidBY - 1) / kResidBY,
            (a.nz + a.kchunk - 1) / a.kchunk);
  // carriers: 0 none, 1 Boltzmann statistics only, 2 with Fermi-Dirac planes
  if (a.coef_df) {
    if (a.carriers == 2) launch_k(resid_kernel<T, 2, true>, grid, block, 0, s, a);
    else if (a.carriers == 1) launch_k(resid_kernel<T, 1, true>, grid, block, 0, s, a);
    else launch_k(resid_kernel<T, 0, true>, grid, block, 0, s, a);
  } else {
    if (a.carriers == 2) launch_k(resid_kernel<T, 2>, grid, block, 0, s, a);
    else if (a.carriers == 1) launch_k(resid_kernel<T, 1>, grid, block, 0, s, a);
    else launch_k(resid_kernel<T, 0>, grid, block, 0, s, a);
  }
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

// the double-float pair routine on arguments given as float pairs (h, l); each
// result pair is returned as its FP64 sum
__global__ void __launch_bounds__(256) carrier_exp_df_kernel(const float2* __restrict__ u,
                                                             double* __restrict__ ep,
                                                             double* __restrict__ em, long long n) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) {
    const float2 v = u[i];
    df a, b;
    exp_pm_df(df{v.x, v.y}, a, b);
    ep[i] = (double)a.h + (double)a.l;
    em[i] = (double)b.h + (double)b.l;
  }
}

cudaError_t launch_carrier_exp_df(const float* u_hl, double* ep, double* em, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  long long b = (n + 255) / 256;
  if (b > 152LL * 8) b = 152LL * 8;
  carrier_exp_df_kernel<<<(int)b, 256, 0, s>>>(reinterpret_cast<const float2*>(u_hl), ep, em, n);
  return cudaGetLastError();
}

#define FX_INST(T)                                                                              \
  template void launch_smooth<T>(const MGArgs<T>&, const LevelDesc&, int, int,                  \
                                 const UpdateArgs*, cudaStream_t, const DevStats*);             \
  template int smooth_rb_tile<T>(const LevelDesc&, bool);                                       \
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

// Per-cell and per-column device functions of the multigrid and of the FP64
// outer residual, shared by the multi-kernel path (multigrid.cu) and the
// persistent batched engine (persistent.cu).  See multigrid.cu for the method.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#include "carrier_exp.cuh"
#include "df_arith.cuh"
#include "ferrox_internal.cuh"

namespace fx {
namespace dev {

// arenas hold fewer than 2^31 elements (checked at init), so 32-bit indices suffice
__device__ __forceinline__ int lidx(const LevelDesc& L, int i, int j, int k) {
  return (int)L.off + (k * L.ny + j) * L.nx + i;
}

// (r + sum of couplings * neighbours) of one cell; the Gauss-Seidel numerator.
template <typename T>
__device__ __forceinline__ T gs_numerator(const T* e, const T* r, const PlaneCoef<T>& c,
                                          const LevelDesc& L, int i, int j, int k, int id) {
  const int im = (i == 0) ? L.nx - 1 : i - 1;
  const int ip = (i == L.nx - 1) ? 0 : i + 1;
  const int jm = (j == 0) ? L.ny - 1 : j - 1;
  const int jp = (j == L.ny - 1) ? 0 : j + 1;
  const int row = id - i;
  const int plane = L.nx * L.ny;
  T sx = e[row + im] + e[row + ip];
  T sy = e[id + (jm - j) * L.nx] + e[id + (jp - j) * L.nx];
  T ed = (k > 0) ? e[id - plane] : T(0);
  T eu = (k < L.nz - 1) ? e[id + plane] : T(0);
  T acc = r[id];
  acc = fma(c.cx, sx, acc);
  acc = fma(c.cy, sy, acc);
  acc = fma(c.czlo, ed, acc);
  acc = fma(c.czhi, eu, acc);
  return acc;
}

struct Upd {
  double* phi;      // fine-level potential (null: no fused update)
  double clamp;     // |e| limit of one update (infinite without carriers)
  int zero;         // set phi = 0 (degenerate zero right-hand side)
  float clampf;     // the limit rounded to FP32 (FP32 corrections)
};

// phi += e, e clamped to [-clamp, clamp].  An FP32 correction is clamped in FP32
// against the limit rounded to float and converted once: one FP64-pipe
// conversion and one FP64 add per cell instead of a conversion, two FP64
// min/max and the add (GB300 runs FP64 at 1/58 of the FP32 rate).  With an
// infinite limit (no carriers) the result is the same bit for bit.
template <typename T>
__device__ __forceinline__ void apply_update(const Upd& u, int idx, T e) {
  if (u.zero) {
    u.phi[idx] = 0.0;
  } else if constexpr (sizeof(T) == sizeof(float)) {
    u.phi[idx] += (double)fminf(fmaxf(e, -u.clampf), u.clampf);
  } else {
    u.phi[idx] += fmin(fmax(e, -u.clamp), u.clamp);
  }
}

// One red/black pair position (ip) of a row: update the cell of `color`; on a
// zero-start sweep also zero the other cell; optionally fold both cells' final
// corrections into phi (last black sweep of the fine level).
template <typename T>
__device__ __forceinline__ void smooth_pair(const MGArgs<T>& a, const LevelDesc& L, int ip, int j,
                                            int k, int color, int zero_init, const Upd& u) {
  const int par = (j + k + color) & 1;
  const int i = 2 * ip + par;
  const int i2 = 2 * ip + (par ^ 1);
  const PlaneCoef<T> c = ldg_struct(a.coef + L.coef_off + k);
  T ev = T(0);
  int id = -1;
  if (i < L.nx) {
    id = lidx(L, i, j, k);
    if (zero_init) {
      const T d = c.has_s ? (a.sinv ? a.sinv[id - L.off] : T(1) / (c.diag + a.s[id])) : c.invdiag;
      ev = a.r[id] * d;
    } else {
      const T num = gs_numerator(a.e, a.r, c, L, i, j, k, id);
      ev = c.has_s ? (a.sinv ? num * a.sinv[id - L.off] : num / (c.diag + a.s[id])) : num * c.invdiag;
    }
    a.e[id] = ev;
  }
  if (i2 < L.nx) {
    const int id2 = lidx(L, i2, j, k);
    if (zero_init) a.e[id2] = T(0);
    if (u.phi) apply_update(u, id2 - L.off, a.e[id2]);
  }
  if (u.phi && id >= 0) apply_update(u, id - L.off, ev);
}

// residual of one fine cell: r - (A + s) e
template <typename T>
__device__ __forceinline__ T cell_residual(const MGArgs<T>& a, const LevelDesc& L, int i, int j,
                                           int k) {
  const PlaneCoef<T> c = ldg_struct(a.coef + L.coef_off + k);
  const int id = lidx(L, i, j, k);
  T num = gs_numerator(a.e, a.r, c, L, i, j, k, id);   // r + couplings * neighbours
  T d = c.has_s ? c.diag + a.s[id] : c.diag;
  return fma(-d, a.e[id], num);
}

// A red/black pre-smoothing ends with the black colour ((i + j + k) odd), whose
// cells were just relaxed against red neighbours that have not changed since:
// their residual is zero up to rounding.  With skip_black set, restriction
// sums the residuals of the red children only (half the arithmetic).  The
// colouring is a proper 2-colouring only if every periodic lateral size is
// even (or 1); black_residual_zero() tells the callers when that holds.
__host__ __device__ __forceinline__ int black_residual_zero(const LevelDesc& F, int nu1) {
  return nu1 > 0 && (F.nx == 1 || !(F.nx & 1)) && (F.ny == 1 || !(F.ny & 1));
}

// Residual of the children of coarse cell (I, J, K) on level F (arrays of `fa`),
// their mean written to the coarse right-hand side rc (and the mean Newton shift
// to sc).  NORM also accumulates the squared residuals of the children it
// computes into rr and, with want_b, the squared right-hand sides of all
// children into bb (the direct FP64 form's stopping test).
//
// With a float accumulator (the direct FP64 form's check) the squares are summed
// in FP32 from FP32 approximations taken with integer operations (the FP64 ->
// FP32 conversion instruction runs on the FP64 pipe): the norms only scale the
// stopping test, where a relative error of ~1e-6 in ||r|| is immaterial.
template <typename T, bool NORM = false, typename A = double>
__device__ __forceinline__ void restrict_children(const MGArgs<T>& fa, T* rc, T* sc,
                                                  const LevelDesc& F, const LevelDesc& C, int I,
                                                  int J, int K, int skip_black, A& rr,
                                                  A& bb, int want_b) {
  const int nxc = F.crx ? 2 : 1, nyc = F.cry ? 2 : 1, nzc = F.crz ? 2 : 1;
  const int i0 = F.crx ? 2 * I : I, j0 = F.cry ? 2 * J : J, k0 = F.crz ? 2 * K : K;
  T sum = T(0), ssum = T(0);
  for (int dk = 0; dk < nzc; ++dk)
    for (int dj = 0; dj < nyc; ++dj)
      for (int di = 0; di < nxc; ++di) {
        const int i = i0 + di, j = j0 + dj, k = k0 + dk;
        if (!(skip_black && ((i + j + k) & 1))) {
          const T r = cell_residual(fa, F, i, j, k);
          sum += r;
          if constexpr (NORM && sizeof(A) == sizeof(float)) {
            const float rf = dev::df_from_double((double)r).h;
            rr = fmaf(rf, rf, rr);
          } else if constexpr (NORM) {
            rr = fma((double)r, (double)r, rr);
          }
        }
        if (NORM && want_b) {
          const double b = fa.r[lidx(F, i, j, k)];
          if constexpr (sizeof(A) == sizeof(float)) {
            const float bf = dev::df_from_double(b).h;
            bb = fmaf(bf, bf, bb);
          } else {
            bb = fma(b, b, bb);
          }
        }
        if (sc) ssum += fa.s[lidx(F, i, j, k)];
      }
  const T inv = T(1) / T(nxc * nyc * nzc);
  const int idc = lidx(C, I, J, K);
  rc[idc] = sum * inv;
  if (sc) sc[idc] = ssum * inv;
}

template <typename T>
__device__ __forceinline__ void restrict_cell(const MGArgs<T>& a, const LevelDesc& F,
                                              const LevelDesc& C, int I, int J, int K,
                                              int skip_black = 0) {
  double rr = 0.0, bb = 0.0;
  restrict_children<T, false>(a, a.r, a.s, F, C, I, J, K, skip_black, rr, bb, 0);
}

// Prolongation + correction for the children of coarse cell (I, J, K).
// Cell-centred trilinear interpolation, separable: along every coarsened
// direction a child takes 3/4 of its own coarse value and 1/4 of the coarse
// neighbour on its side; an electrode beyond the coarse grid acts as a ghost
// cell holding -e (zero correction on the electrode face).
template <typename T>
__device__ __forceinline__ void prolong_cell(const MGArgs<T>& a, const LevelDesc& F,
                                             const LevelDesc& C, int I, int J, int K, int constant) {
  const int nxc = F.crx ? 2 : 1, nyc = F.cry ? 2 : 1, nzc = F.crz ? 2 : 1;
  T* e = a.e;
  if (constant) {
    const T E0 = e[lidx(C, I, J, K)];
    for (int c = 0; c < nzc; ++c)
      for (int b = 0; b < nyc; ++b)
        for (int q = 0; q < nxc; ++q)
          e[lidx(F, F.crx ? 2 * I + q : I, F.cry ? 2 * J + b : J, F.crz ? 2 * K + c : K)] += E0;
    return;
  }
  const int Im = I == 0 ? C.nx - 1 : I - 1, Ip = I + 1 == C.nx ? 0 : I + 1;
  const int Jm = J == 0 ? C.ny - 1 : J - 1, Jp = J + 1 == C.ny ? 0 : J + 1;
  const int xs[3] = {Im, I, Ip}, ys[3] = {Jm, J, Jp};
  T Z[2][3][3];
#pragma unroll
  for (int yy = 0; yy < 3; ++yy)
#pragma unroll
    for (int xx = 0; xx < 3; ++xx) {
      if ((!F.cry && yy != 1) || (!F.crx && xx != 1)) continue;
      const T Ec = e[lidx(C, xs[xx], ys[yy], K)];
      if (F.crz) {
        Z[0][yy][xx] = (K > 0) ? fma(T(0.75), Ec, T(0.25) * e[lidx(C, xs[xx], ys[yy], K - 1)])
                               : T(0.5) * Ec;
        Z[1][yy][xx] = (K + 1 < C.nz) ? fma(T(0.75), Ec, T(0.25) * e[lidx(C, xs[xx], ys[yy], K + 1)])
                                      : T(0.5) * Ec;
      } else {
        Z[0][yy][xx] = Ec;
      }
    }
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    if (c >= nzc) break;
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      if (b >= nyc) break;
      T Y[3];
#pragma unroll
      for (int xx = 0; xx < 3; ++xx) {
        if (!F.crx && xx != 1) continue;
        Y[xx] = F.cry ? fma(T(0.75), Z[c][1][xx], T(0.25) * Z[c][b ? 2 : 0][xx]) : Z[c][1][xx];
      }
      const int fj = F.cry ? 2 * J + b : J, fk = F.crz ? 2 * K + c : K;
      if (F.crx) {
        const int f0 = lidx(F, 2 * I, fj, fk);
        e[f0] += fma(T(0.75), Y[1], T(0.25) * Y[0]);
        e[f0 + 1] += fma(T(0.75), Y[1], T(0.25) * Y[2]);
      } else {
        e[lidx(F, I, fj, fk)] += Y[1];
      }
    }
  }
}

// Prolongation + correction of one fine cell (i, j, k) of F: the separable
// trilinear interpolation of prolong_cell (z, then y, then x, the same
// operations in the same order), evaluated per fine cell, so that a tiny level
// spreads its arithmetic over one thread per fine cell.
template <typename T>
__device__ __forceinline__ void prolong_fine(const MGArgs<T>& a, const LevelDesc& F,
                                             const LevelDesc& C, int i, int j, int k,
                                             int constant) {
  T* e = a.e;
  const int I = F.crx ? i >> 1 : i, J = F.cry ? j >> 1 : j, K = F.crz ? k >> 1 : k;
  if (constant) {
    e[lidx(F, i, j, k)] += e[lidx(C, I, J, K)];
    return;
  }
  // the coarse neighbour on the child's side in each coarsened direction
  const int I2 = !F.crx ? I : (i & 1) ? (I + 1 == C.nx ? 0 : I + 1) : (I == 0 ? C.nx - 1 : I - 1);
  const int J2 = !F.cry ? J : (j & 1) ? (J + 1 == C.ny ? 0 : J + 1) : (J == 0 ? C.ny - 1 : J - 1);
  const int K2 = (k & 1) ? K + 1 : K - 1;   // outside [0, C.nz): electrode ghost (-e)
  auto zcol = [&](int x, int y) -> T {
    const T c0 = e[lidx(C, x, y, K)];
    if (!F.crz) return c0;
    return (K2 >= 0 && K2 < C.nz) ? fma(T(0.75), c0, T(0.25) * e[lidx(C, x, y, K2)])
                                  : T(0.5) * c0;
  };
  const T z11 = zcol(I, J);
  T y1 = z11, y2 = T(0);
  if (F.cry) y1 = fma(T(0.75), z11, T(0.25) * zcol(I, J2));
  if (F.crx) {
    const T z21 = zcol(I2, J);
    y2 = F.cry ? fma(T(0.75), z21, T(0.25) * zcol(I2, J2)) : z21;
    e[lidx(F, i, j, k)] += fma(T(0.75), y1, T(0.25) * y2);
  } else {
    e[lidx(F, i, j, k)] += y1;
  }
}

// ---- single-CTA tail: the smallest levels in shared memory ---------------------------

// Division by a level constant d without the integer divide sequence: with
// m = ceil(2^32 / d) = floor((2^32 - 1) / d) + 1 (one 32-bit divide per call),
// floor(t m / 2^32) = floor(t / d) for all t < 2^16 and d <= 2^16 (Granlund and
// Montgomery, PLDI 1994: the error t (m d - 2^32) / d stays below 2^32 / d).
// The tail's shared-memory budget keeps every tail level below 2^16 cells, so
// all indices of a tail sweep are in range.
static_assert(kTailMaxSmem / (2 * sizeof(float)) < 65536, "tail indices must stay below 2^16");

__device__ __forceinline__ unsigned long long magic32(unsigned d) {
  return (unsigned long long)(0xFFFFFFFFu / d) + 1ull;
}
__device__ __forceinline__ int div32(int t, unsigned long long m) {
  return (int)(((unsigned long long)(unsigned)t * m) >> 32);
}

// FX_TAIL_LINKAGE: how tail_smooth and tail_vcycle are compiled in this
// translation unit.  The batched engines (persistent.cu) set __noinline__:
// inlined there, the FP64 instantiation lost the tail's smoothing (the first
// tail level kept its old shared-memory contents; 35 V-cycles per solve instead
// of 8 on a 32x32x16 stack), depending only on the surrounding code.  The
// single-instance tail kernel inlines them (same V-cycle counts either way,
// checked by the solver tests' cycle bounds).
#ifndef FX_TAIL_LINKAGE
#define FX_TAIL_LINKAGE
#endif
template <typename T>
__device__ FX_TAIL_LINKAGE void tail_smooth(const MGArgs<T>& a, const LevelDesc& L, int sweeps, int zero_first) {
  const int hx = (L.nx + 1) >> 1;
  const int items = hx * L.ny * L.nz;
  const unsigned long long mx = magic32(hx), my = magic32(L.ny);
  const Upd none{nullptr, 0.0, 0, 0.0f};
  for (int sw = 0; sw < sweeps; ++sw)
    for (int color = 0; color < 2; ++color) {
      const int zi = (zero_first && sw == 0 && color == 0);
      for (int t = threadIdx.x; t < items; t += blockDim.x) {
        const int rest = div32(t, mx), k = div32(rest, my);
        smooth_pair(a, L, t - rest * hx, rest - k * L.ny, k, color, zi, none);
      }
      __syncthreads();
    }
}

// e = A^-1 r on a level of n <= kDenseMax cells: the inverse (row-major, computed
// on the host in FP64) times r, four lanes per row and a fixed-order reduction.
template <typename T>
__device__ void tail_dense(const T* __restrict__ inv, int n, const T* r, T* e) {
  const int tid = threadIdx.x;
  if ((tid >> 5) < ((4 * n + 31) >> 5)) {   // whole warps, for the shuffles
    const int row = tid >> 2, p = tid & 3;
    T acc = T(0);
    if (row < n)
      for (int c = p; c < n; c += 4) acc = fma(__ldg(inv + row * n + c), r[c], acc);
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    if (row < n && p == 0) e[row] = acc;
  }
  __syncthreads();
}

// A complete V-cycle over the tail levels of one instance, by one CTA, with the
// level arrays in shared memory (smem holds 2 or 3 arrays of t.elems values).
// With t.dense the level t.dense_lev is solved exactly by its inverse and the
// levels below it are not visited; otherwise the coarsest level is relaxed
// t.bottom_sweeps times.
template <typename T>
__device__ FX_TAIL_LINKAGE void tail_vcycle(const MGArgs<T>& g, const TailArgs& t, unsigned char* tail_smem) {
  T* se = reinterpret_cast<T*>(tail_smem);
  T* sr = se + t.elems;
  T* ss = g.s ? sr + t.elems : nullptr;
  const LevelDesc* lv = t.lv;
  const int n0 = (int)lv[0].ncell;
  for (int q = threadIdx.x; q < n0; q += blockDim.x) {
    sr[q] = g.r[t.base + q];
    if (ss) ss[q] = g.s[t.base + q];
  }
  __syncthreads();
  MGArgs<T> a;
  a.e = se; a.r = sr; a.s = ss; a.coef = g.coef; a.lv = lv;
  const int bottom = t.dense ? t.dense_lev : t.nlev - 1;
  for (int l = 0; l < bottom; ++l) {
    const LevelDesc F = ldg_struct(lv + l), C = ldg_struct(lv + l + 1);
    tail_smooth(a, F, t.nu1, 1);
    const int nc = (int)C.ncell;
    const unsigned long long mx = magic32(C.nx), my = magic32(C.ny);
    const int skip = black_residual_zero(F, t.nu1);
    for (int q = threadIdx.x; q < nc; q += blockDim.x) {
      const int rest = div32(q, mx), K = div32(rest, my);
      restrict_cell(a, F, C, q - rest * C.nx, rest - K * C.ny, K, skip);
    }
    __syncthreads();
  }
  if (t.dense) {
    const LevelDesc B = ldg_struct(lv + bottom);
    tail_dense(static_cast<const T*>(t.dense), (int)B.ncell, sr + B.off, se + B.off);
  } else {
    tail_smooth(a, lv[bottom], t.bottom_sweeps, 1);
  }
  for (int l = bottom - 1; l >= 0; --l) {
    const LevelDesc F = ldg_struct(lv + l), C = ldg_struct(lv + l + 1);
    const int nf = (int)F.ncell;
    const unsigned long long mx = magic32(F.nx), my = magic32(F.ny);
    for (int q = threadIdx.x; q < nf; q += blockDim.x) {
      const int rest = div32(q, mx), k = div32(rest, my);
      prolong_fine(a, F, C, q - rest * F.nx, rest - k * F.ny, k, t.constant);
    }
    __syncthreads();
    tail_smooth(a, F, t.nu2, 0);
  }
  for (int q = threadIdx.x; q < n0; q += blockDim.x) g.e[t.base + q] = se[q];
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block sum of one value; result valid in thread 0.
__device__ __forceinline__ void block_sum1(double& x) {
  __shared__ double sh1[32];
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int nthr = blockDim.x * blockDim.y;
  x = warp_sum(x);
  const int w = tid >> 5, l = tid & 31;
  if (l == 0) sh1[w] = x;
  __syncthreads();
  if (w == 0) x = warp_sum(l < ((nthr + 31) >> 5) ? sh1[l] : 0.0);
  __syncthreads();
}

// Block sum of three values; result valid in thread 0.
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// FP32 block sums of two per-thread values (the double-float residual's norms, which
// decide a tolerance: FP32 sums within a block are ample); valid in thread 0
__device__ __forceinline__ void block_sum2f(float& x, float& y) {
  __shared__ float shf[2][32];
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int nthr = blockDim.x * blockDim.y;
  x = warp_sum_f(x); y = warp_sum_f(y);
  const int w = tid >> 5, l = tid & 31;
  if (l == 0) { shf[0][w] = x; shf[1][w] = y; }
  __syncthreads();
  const int nw = (nthr + 31) >> 5;
  if (w == 0) {
    x = l < nw ? shf[0][l] : 0.0f;
    y = l < nw ? shf[1][l] : 0.0f;
    x = warp_sum_f(x); y = warp_sum_f(y);
  }
  __syncthreads();
}

__device__ __forceinline__ void block_sum3(double& x, double& y, double& z) {
  __shared__ double sh[3][32];
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int nthr = blockDim.x * blockDim.y;
  x = warp_sum(x); y = warp_sum(y); z = warp_sum(z);
  const int w = tid >> 5, l = tid & 31;
  if (l == 0) { sh[0][w] = x; sh[1][w] = y; sh[2][w] = z; }
  __syncthreads();
  const int nw = (nthr + 31) >> 5;
  if (w == 0) {
    x = l < nw ? sh[0][l] : 0.0;
    y = l < nw ? sh[1][l] : 0.0;
    z = l < nw ? sh[2][l] : 0.0;
    x = warp_sum(x); y = warp_sum(y); z = warp_sum(z);
  }
  __syncthreads();
}

// FP64 -> FP32 store of the outer residual (mixed form) by integer truncation:
// sign, rebiased exponent and the top 23 mantissa bits, rounding toward zero
// (within 1 FP32 ulp; the FP64 defect correction absorbs it).  Magnitudes below
// the FP32 normal range store a signed zero, above it (and NaN) infinity; the
// norms and the convergence decision use the FP64 value.  The conversion
// instruction would run on the FP64 pipe that bounds this kernel.
template <typename T>
__device__ __forceinline__ T narrow_resid(double x) {
  if (sizeof(T) == sizeof(float)) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    const int e = (int)((b >> 52) & 0x7ff) - 1023 + 127;
    if (e <= 0) return (T)__uint_as_float(sign);
    if (e >= 255) return (T)__uint_as_float(sign | 0x7f800000u);
    return (T)__uint_as_float(sign | ((unsigned)e << 23) | (unsigned)((b >> 29) & 0x7fffffu));
  }
  return (T)x;
}

// Fermi-Dirac integral of order 1/2 (normalised to e^eta for eta -> -inf) and its
// derivative, by the approximation of Bednarczyk & Bednarczyk (1978) that the paper
// uses for the carrier integrals: F = 1/(e^-eta + xi), xi = (3 sqrt(pi)/4) v^(-3/8),
// v = eta^4 + 50 + 33.6 eta (1 - 0.68 e^(-0.17 (eta + 1)^2)).  Far below the band
// edge (eta < -700, where e^-eta overflows) F = e^eta to double precision.
__device__ __forceinline__ double fd_half(double eta, double& dF) {
  if (eta < -700.0) {
    dF = exp(eta);
    return dF;
  }
  const double g = exp(-0.17 * (eta + 1.0) * (eta + 1.0));
  const double w = fma(-0.68, g, 1.0);
  const double e2 = eta * eta;
  const double v = fma(e2, e2, fma(33.6 * eta, w, 50.0));
  const double dv = fma(4.0 * e2, eta, 33.6 * fma(eta * 0.2312 * g, eta + 1.0, w));
  const double xi = 1.3293403881791355 * exp(-0.375 * log(v));   // (3 sqrt(pi)/4) v^(-3/8)
  const double dxi = -0.375 * xi * dv / v;
  const double em = exp(-eta);
  const double F = 1.0 / (em + xi);
  dF = (em - dxi) * F * F;
  return F;
}

// FP64 residual of planes [k0, k1) of one (x, y) column, marching up with a
// register window; accumulates r^2, b^2 (first residual of a solve only) and
// rho^2.  SC = 0 compiles out the carrier term (stacks without a semiconductor
// layer), SC = 1 keeps Boltzmann statistics only, SC = 2 also Fermi-Dirac.
// The Newton shift of a level-0 cell, and with sinv_out the reciprocal of the
// shifted diagonal (in T, from the diagonal as the sweeps' T coefficients hold
// it), which the level-0 sweeps multiply by instead of dividing in every sweep.
template <typename T>
__device__ __forceinline__ void put_shift(const ResidArgs& a, long long t, double sv, T diag_t) {
  const T s = (T)sv;
  static_cast<T*>(a.s_out)[t] = s;
  if (a.sinv_out) static_cast<T*>(a.sinv_out)[t] = T(1) / (diag_t + s);
}

// the level-0 diagonal in T from its double-float pair (float: the high part is
// the nearest float)
template <typename T>
__device__ __forceinline__ T diag_of_df(const PlaneCoefDF& c) {
  if constexpr (sizeof(T) == sizeof(float)) return c.diag_h;
  else return (double)c.diag_h + (double)c.diag_l;
}

template <typename T, int SC = 2>
__device__ __forceinline__ void resid_column(const ResidArgs& a, int i, int j, int k0, int k1,
                                             double& acc_r, double& acc_b, double& acc_rho) {
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const long long plane = (long long)nx * ny;
  T* r_out = static_cast<T*>(a.r_out);
  T* s_out = static_cast<T*>(a.s_out);
  const double v_bot = a.params->v_bot, v_top = a.params->v_top;
  const int im = (i == 0) ? nx - 1 : i - 1, ip = (i == nx - 1) ? 0 : i + 1;
  const long long dxm = im - i, dxp = ip - i;
  const long long dym = (long long)((j == 0) ? ny - 1 : j - 1) * nx - (long long)j * nx;
  const long long dyp = (long long)((j == ny - 1) ? 0 : j + 1) * nx - (long long)j * nx;
  const double* phi = a.phi;
  const long long col = (long long)j * nx + i;
  double pd = k0 > 0 ? phi[(long long)(k0 - 1) * plane + col] : 0.0;
  double pc = phi[(long long)k0 * plane + col];
  for (int k = k0; k < k1; ++k) {
    const long long t = k * plane + col;
    const double pu = (k < nz - 1) ? phi[t + plane] : 0.0;
    const PlaneCoef<double> c = ldg_struct(a.coef0 + k);
    const PlaneTDGL pt = ldg_struct(a.planes + k);
    const double sx = phi[t + dxm] + phi[t + dxp];
    const double sy = phi[t + dym] + phi[t + dyp];
    double bb;
    if (pt.b_dyn) {
      bb = a.b[t];
    } else {
      bb = 0.0;
      if (k == 0) bb += pt.lift * v_bot;
      if (k == nz - 1) bb += pt.lift * v_top;
    }
    double rho = 0.0;
    if (SC && pt.sc) {
      if (SC == 2 && pt.fd) {
        // n = Nc F(eta_e0 + u), p = Nv F(eta_p0 - u); -d rho/d phi = kq (dn + dp)/VT
        const double u = pc * pt.inv_vt;
        double dn, dp;
        const double n = pt.Nc * fd_half(pt.eta_e0 + u, dn);
        const double p = pt.Nv * fd_half(pt.eta_p0 - u, dp);
        rho = pt.kq * (p - n + pt.Nnet);
        if (s_out) put_shift<T>(a, t, pt.kq * fma(pt.Nc, dn, pt.Nv * dp) * pt.inv_vt, (T)c.diag);
      } else {
        double ep, em;
        exp_pm(pc * pt.inv_vt, ep, em);
        const double n = pt.n0 * ep;
        const double p = pt.p0 * em;
        rho = pt.kq * (p - n + pt.Nnet);
        if (s_out) put_shift<T>(a, t, pt.kq * (n + p) * pt.inv_vt, (T)c.diag);
      }
      acc_rho = fma(rho, rho, acc_rho);
    }
    // r = b + rho - A phi = (b + rho) - diag phi + couplings * neighbours
    double r = fma(-c.diag, pc, SC ? bb + rho : bb);
    r = fma(c.czhi, pu, r);
    r = fma(c.czlo, pd, r);
    r = fma(c.cy, sy, r);
    r = fma(c.cx, sx, r);
    r_out[t] = narrow_resid<T>(r);
    acc_r = fma(r, r, acc_r);
    if (a.first) acc_b = fma(bb, bb, acc_b);
    pd = pc;
    pc = pu;
  }
}

// The same residual with the stencil in double-float arithmetic (df_arith.cuh):
// the potentials, the right-hand side b + rho and the coefficients enter as h + l
// pairs, the products and sums keep about 48 bits, so r agrees with the FP64
// residual to a few 2^-48 of the largest term while the FP64 pipe is left to the
// carrier exponentials.  The output is the high part (T = float, the mixed form's
// FP32 correction equation) or h + l (T = double); the squared norms accumulate
// per thread in FP32 (they decide a tolerance, 1e-7 relative is ample) and enter
// the block sums in FP64.
template <typename T, int SC>
__device__ __forceinline__ void resid_column_df(const ResidArgs& a, int i, int j, int k0, int k1,
                                                float& acc_r, float& acc_b, double& acc_rho) {
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const long long plane = (long long)nx * ny;
  T* r_out = static_cast<T*>(a.r_out);
  T* s_out = static_cast<T*>(a.s_out);
  const double v_bot = a.params->v_bot, v_top = a.params->v_top;
  const int im = (i == 0) ? nx - 1 : i - 1, ip = (i == nx - 1) ? 0 : i + 1;
  const long long dxm = im - i, dxp = ip - i;
  const long long dym = (long long)((j == 0) ? ny - 1 : j - 1) * nx - (long long)j * nx;
  const long long dyp = (long long)((j == ny - 1) ? 0 : j + 1) * nx - (long long)j * nx;
  const double* phi = a.phi;
  const long long col = (long long)j * nx + i;
  double pc_d = phi[(long long)k0 * plane + col];
  df pd = k0 > 0 ? df_from_double(phi[(long long)(k0 - 1) * plane + col]) : df{0.0f, 0.0f};
  df pc = df_from_double(pc_d);
  float rho2f = 0.0f;   // rho^2 of the double-float carrier path (enters only the scale of the test)
  for (int k = k0; k < k1; ++k) {
    const long long t = k * plane + col;
    const double pu_d = (k < nz - 1) ? phi[t + plane] : 0.0;
    const df pu = df_from_double(pu_d);
    const PlaneCoefDF c = ldg_struct(a.coef_df + k);
    // only the plane fields this cell needs (the whole record is 28 words)
    const PlaneTDGL* pk = a.planes + k;
    const int b_dyn = __ldg(&pk->b_dyn);
    // x neighbours: the centre pairs of the neighbouring lanes when a warp holds 32
    // cells of one row (the row's ends convert their own)
    df xm, xp;
    if (a.warp_rows) {
      const int lane = threadIdx.x & 31;
      xm.h = __shfl_up_sync(0xffffffffu, pc.h, 1);
      xm.l = __shfl_up_sync(0xffffffffu, pc.l, 1);
      xp.h = __shfl_down_sync(0xffffffffu, pc.h, 1);
      xp.l = __shfl_down_sync(0xffffffffu, pc.l, 1);
      if (lane == 0) xm = df_from_double(phi[t + dxm]);
      if (lane == 31) xp = df_from_double(phi[t + dxp]);
    } else {
      xm = df_from_double(phi[t + dxm]);
      xp = df_from_double(phi[t + dxp]);
    }
    const df sx = df_add_fast(xm, xp);
    const df sy = df_add_fast(df_from_double(phi[t + dym]), df_from_double(phi[t + dyp]));
    double bb;
    if (b_dyn) {
      bb = a.b[t];
    } else {
      bb = 0.0;
      if (k == 0) bb += __ldg(&pk->lift) * v_bot;
      if (k == nz - 1) bb += __ldg(&pk->lift) * v_top;
    }
    df b_df = df_from_double(bb);
    if (SC && __ldg(&pk->sc)) {
      const PlaneTDGL pt = ldg_struct(pk);
      // Boltzmann densities in double-float on the FP32 pipe while |u| <= kExpDFMax:
      // rho = kq p0 e^{-u} - kq n0 e^{u} + kq Nnet, u = phi / V_T
      const df inv_vt = df_from_double(pt.inv_vt);
      const df u = df_mul(pc, inv_vt);
      if (!(SC == 2 && pt.fd) && fabsf(u.h) <= kExpDFMax) {
        df ep, em;
        exp_pm_df(u, ep, em);
        const df kn = df_mul(df_from_double(pt.kqn0), ep);
        const df kp = df_mul(df_from_double(pt.kqp0), em);
        const df rho = df_add(df_add(kp, df_neg(kn)), df_from_double(pt.kqN));
        b_df = df_add(b_df, rho);
        rho2f = fmaf(rho.h, rho.h, rho2f);
        if (s_out) {
          const float sv = (kn.h + kp.h) * inv_vt.h;
          s_out[t] = (T)sv;
          if (a.sinv_out) static_cast<T*>(a.sinv_out)[t] = (T)(1.0f / (c.diag_h + sv));
        }
      } else {
        double rho;
        if (SC == 2 && pt.fd) {
          const double uu = pc_d * pt.inv_vt;
          double dn, dp;
          const double n = pt.Nc * fd_half(pt.eta_e0 + uu, dn);
          const double p = pt.Nv * fd_half(pt.eta_p0 - uu, dp);
          rho = pt.kq * (p - n + pt.Nnet);
          if (s_out) put_shift<T>(a, t, pt.kq * fma(pt.Nc, dn, pt.Nv * dp) * pt.inv_vt, diag_of_df<T>(c));
        } else {
          double ep, em;
          exp_pm(pc_d * pt.inv_vt, ep, em);
          const double n = pt.n0 * ep;
          const double p = pt.p0 * em;
          rho = pt.kq * (p - n + pt.Nnet);
          if (s_out) put_shift<T>(a, t, pt.kq * (n + p) * pt.inv_vt, diag_of_df<T>(c));
        }
        b_df = df_from_double(bb + rho);
        acc_rho = fma(rho, rho, acc_rho);
      }
    }
    // r = ((b + rho) - diag phi) + (z couplings) + (lateral couplings), as a tree
    const df r0 = df_add_fast(b_df, df_neg(df_mul(df{c.diag_h, c.diag_l}, pc)));
    const df rz = df_add_fast(df_mul(df{c.czhi_h, c.czhi_l}, pu), df_mul(df{c.czlo_h, c.czlo_l}, pd));
    const df rl = df_add_fast(df_mul(df{c.cy_h, c.cy_l}, sy), df_mul(df{c.cx_h, c.cx_l}, sx));
    const df r = df_add_fast(df_add_fast(r0, rz), rl);
    if (sizeof(T) == sizeof(float))
      r_out[t] = (T)r.h;
    else
      r_out[t] = (T)((double)r.h + (double)r.l);
    acc_r = fmaf(r.h, r.h, acc_r);
    if (a.first) {
      const float bh = df_from_double(bb).h;
      acc_b = fmaf(bh, bh, acc_b);
    }
    pd = pc;
    pc = pu;
    pc_d = pu_d;
  }
  if (SC) acc_rho += (double)rho2f;
}

// Convergence decision of one solve from its summed norms (one thread).
__device__ __forceinline__ int decide(DevStats* st, double sr, double sb, double sq, int first,
                                      double tol, int max_cycles, int launches_per_cycle,
                                      int adapt_max = 0, int launches_per_vcycle = 0,
                                      int inner_fixed = 1) {
  if (first) {
    st->solves += 1;
    st->cycles_this_solve = 0;
    st->zero_phi = 0;
    st->launches += 1;
    st->bnorm2 = sb;          // b is fixed during a solve
  }
  const double rn = sqrt(sr);
  const double scale = fmax(sqrt(st->bnorm2), sqrt(sq));
  int cond;
  if (!isfinite(rn) || !isfinite(scale)) {
    if (st->status == 0) st->status = FERROX_ENONFINITE;
    cond = 0;
  } else if (rn <= tol * scale) {
    cond = 0;
  } else if (st->cycles_this_solve >= max_cycles) {
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
    st->launches += launches_per_cycle;
    if (adapt_max <= 0) st->vcycles += inner_fixed;
  }
  if (adapt_max > 0 && !first && st->inner_k > 0 && st->prev_rnorm > 0.0 && rn > 0.0) {
    // contraction per V-cycle over the outer iteration just finished, measured
    // whether or not it reached the tolerance (kept for the next solves)
    st->rho_v = fmin(fmax(pow(rn / st->prev_rnorm, 1.0 / st->inner_k), 0.02), 0.9);
  }
  if (cond && adapt_max > 0) {
    // V-cycles for the next outer iteration: enough, at the estimated contraction
    // (0.2 before any measurement), to bring ||r|| to the tolerance
    const double rho = st->rho_v > 0.0 ? st->rho_v : 0.2;
    const double need = (rn > 0.0 && scale > 0.0) ? log(tol * scale / rn) / log(rho) : 1.0;
    const int k = (int)fmin(fmax(ceil(need), 1.0), (double)adapt_max);
    st->inner_k = k;
    st->inner_left = k;
    st->prev_rnorm = rn;
    st->launches += k * launches_per_vcycle;
    st->vcycles += k;
  }
  st->last_cond = cond;
  st->last_cycles = st->cycles_this_solve;
  st->last_rnorm = rn;
  st->last_scale = scale;
  st->last_rel = scale > 0.0 ? rn / scale : (rn > 0.0 ? INFINITY : 0.0);
  return cond;
}

}  // namespace dev
}  // namespace fx

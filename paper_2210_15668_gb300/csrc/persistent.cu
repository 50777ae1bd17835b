// Persistent batched engine: many independent device stacks (a Q-V sweep of
// instances with uneven lateral sizes and biases) advanced by ONE cooperative
// kernel launch.
//
// The CTAs form groups, each owning a contiguous range of instances (one group
// holding every instance and CTA is the plain grid form).  Every phase of the
// time step (TDGL update, FP64 residual, per-instance convergence decision, each
// multigrid level's sweeps and transfers, the shared-memory tail) runs over the
// work units of the group's instances; the phases are separated by the group's
// barrier, so groups advance independently.  Each instance decides its own
// convergence and drops out of the remaining cycles when done.  Work units are
// rows (or `rows_per_unit` consecutive rows) of one plane of one instance,
// handled by one warp whose lanes run along x; the unit -> instance map is a
// binary search in per-phase prefix tables.  Barrier waits are bounded in time:
// on expiry the kernel records FERROX_ETIMEOUT and every block leaves after at
// most one more bounded wait, so a fault elsewhere can never hang the GPU.
#include <cuda_runtime.h>

#include <vector>

#include "ferrox_internal.cuh"
#ifndef FX_TAIL_LINKAGE
#define FX_TAIL_LINKAGE __noinline__   // see mg_device.cuh
#endif
#include "mg_device.cuh"
#include "tdgl_device.cuh"

namespace fx {

namespace {

using namespace dev;

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned int atom_add_acq_rel(unsigned int* p, unsigned int v) {
  unsigned int old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

__device__ __forceinline__ void st_release(unsigned int* p, unsigned int v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier with a time limit.  Returns false (and records the status)
// when the wait ran out or another block has already aborted.
__device__ bool grid_barrier(GridBar* gb, int* status, unsigned int nblocks,
                             long long limit = kBarrierSpinCycles, int* dbg = nullptr,
                             int nbar = 0) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    __threadfence();
    const unsigned int gen = ld_acquire(&gb->gen);
    if (atom_add_acq_rel(&gb->count, 1u) == nblocks - 1) {
      gb->count = 0;
      st_release(&gb->gen, gen + 1);
    } else {
      const long long t0 = clock64();
      while (ld_acquire(&gb->gen) == gen) {
        if (ld_acquire(&gb->abort)) { ok = 0; break; }
        if (clock64() - t0 > limit) {
          if (dbg && atomicCAS(&dbg[0], 0, 1) == 0) {   // where the first wait ran out
            dbg[1] = nbar;
            dbg[2] = (int)blockIdx.x;
            dbg[3] = (int)ld_acquire(&gb->count);
            dbg[4] = (int)gen;
          }
          atomicCAS(status, 0, (int)FERROX_ETIMEOUT);
          st_release(&gb->abort, 1u);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    if (ok && ld_acquire(&gb->abort)) ok = 0;
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

__device__ __forceinline__ int find_inst(const int* pre, int n, int u) {
  int lo = 0, hi = n;   // pre[lo] <= u < pre[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (pre[mid] <= u) lo = mid; else hi = mid;
  }
  return lo;
}

// control flags written by other CTAs of this launch: read at L2
__device__ __forceinline__ int ld_flag(const int* p) { return __ldcg(p); }

// Warp-level sum (all lanes active), result in every lane.
__device__ __forceinline__ double wsum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// A CTA group advances its own instances [i_lo, i_hi) with its own barrier; the
// warps of the group (gwarp of nwarps) share each phase's work units.
template <typename T>
struct Ctx {
  const BatchArgs& A;
  MGArgs<T> mg;
  int lane, gwarp, nwarps;
  int i_lo, i_hi;       // the group's instances
  int grank, ncta;      // this CTA's rank in the group, the group's CTAs
};

// ---- phases -----------------------------------------------------------------------------

// TDGL update (or right-hand side only) of every active column: unit = one row.
template <typename T>
__device__ void phase_tdgl(const Ctx<T>& c, int mode) {
  const BatchArgs& A = c.A;
  const int* pre = A.pre;   // space 0: rows
  const int total = pre[c.i_hi];
  for (int u = pre[c.i_lo] + c.gwarp; u < total; u += c.nwarps) {
    const int i = find_inst(pre, A.ninst, u);
    const BatchInst I = ldg_struct(A.inst + i);
    TDGLArgs t = I.tdgl;
    t.mode = mode;
    const int j = u - pre[i];
    for (int x = c.lane; x < t.nx; x += 32) tdgl_column(t, x, j);
  }
}

// FP64 residual of every active instance; copies the new P back first (order 1).
template <typename T>
__device__ void phase_resid(const Ctx<T>& c, int first, int copy_back) {
  const BatchArgs& A = c.A;
  const int* pre = A.pre;
  const int total = pre[c.i_hi];
  for (int u = pre[c.i_lo] + c.gwarp; u < total; u += c.nwarps) {
    const int i = find_inst(pre, A.ninst, u);
    if (!ld_flag(A.active + i)) continue;
    const BatchInst I = ldg_struct(A.inst + i);
    const int j = u - pre[i];
    ResidArgs ra = I.resid;
    ra.first = first;
    double ar = 0.0, ab = 0.0, aq = 0.0;
    const long long plane = (long long)ra.nx * ra.ny;
    for (int x = c.lane; x < ra.nx; x += 32) {
      if (copy_back) {
        for (int k = I.fe_lo; k <= I.fe_hi; ++k) {
          const long long t = k * plane + (long long)j * ra.nx + x;
          I.P[t] = I.Pbuf[t];
        }
      }
      if (ra.carriers) resid_column<T>(ra, x, j, 0, ra.nz, ar, ab, aq);
      else resid_column<T, 0>(ra, x, j, 0, ra.nz, ar, ab, aq);   // no b + rho add
    }
    ar = wsum(ar); ab = wsum(ab); aq = wsum(aq);
    if (c.lane == 0) {
      A.partials[3 * u] = ar;
      A.partials[3 * u + 1] = ab;
      A.partials[3 * u + 2] = aq;
    }
  }
}

// Per-instance convergence decision: one warp per instance, fixed-order sums.
template <typename T>
__device__ void phase_decide(const Ctx<T>& c, int first) {
  const BatchArgs& A = c.A;
  for (int i = c.i_lo + c.gwarp; i < c.i_hi; i += c.nwarps) {
    if (!ld_flag(A.active + i)) continue;
    double sr = 0.0, sb = 0.0, sq = 0.0;
    for (int u = A.pre[i] + c.lane; u < A.pre[i + 1]; u += 32) {
      sr += A.partials[3 * u];
      sb += A.partials[3 * u + 1];
      sq += A.partials[3 * u + 2];
    }
    sr = wsum(sr); sb = wsum(sb); sq = wsum(sq);
    if (c.lane == 0) {
      const int cond = decide(A.inst[i].resid.stats, sr, sb, sq, first, A.tol, A.max_cycles, 0);
      A.active[i] = cond;
    }
  }
}

// The cells of `color` at pair position ip of rows j0 .. j0+nr-1 (nr <= 4) of plane k:
// smooth_pair's operations, cell by cell in the same order (so the results are
// identical), with the plane's coefficients passed in and every load of the rows
// issued before the first store.  Reordering is safe: a cell of this colour reads
// only cells of the other colour, which this sweep writes only on a zero start,
// where no neighbour is read.
template <typename T>
__device__ __forceinline__ void smooth_rows(const MGArgs<T>& a, const LevelDesc& L, const PlaneCoef<T>& cf,
                                            int ip, int j0, int nr, int k, int color, int zero_init,
                                            const Upd& u) {
  T num[4], sv[4];
  int id[4];
#pragma unroll
  for (int rr = 0; rr < 4; ++rr) {
    id[rr] = -1;
    num[rr] = T(0);
    sv[rr] = T(0);
    if (rr < nr) {
      const int j = j0 + rr;
      const int i = 2 * ip + ((j + k + color) & 1);
      if (i < L.nx) {
        const int t = lidx(L, i, j, k);
        id[rr] = t;
        num[rr] = zero_init ? a.r[t] : gs_numerator(a.e, a.r, cf, L, i, j, k, t);
        if (cf.has_s && !a.sinv) sv[rr] = a.s[t];
      }
    }
  }
#pragma unroll
  for (int rr = 0; rr < 4; ++rr) {
    if (rr >= nr) break;
    const int j = j0 + rr;
    const int i2 = 2 * ip + (((j + k + color) & 1) ^ 1);
    const int t = id[rr];
    T ev = T(0);
    if (t >= 0) {
      if (zero_init) {
        const T d = cf.has_s ? (a.sinv ? a.sinv[t - L.off] : T(1) / (cf.diag + sv[rr])) : cf.invdiag;
        ev = num[rr] * d;
      } else {
        ev = cf.has_s ? (a.sinv ? num[rr] * a.sinv[t - L.off] : num[rr] / (cf.diag + sv[rr]))
                      : num[rr] * cf.invdiag;
      }
      a.e[t] = ev;
    }
    if (i2 < L.nx) {
      const int id2 = lidx(L, i2, j, k);
      if (zero_init) a.e[id2] = T(0);
      if (u.phi) apply_update(u, id2 - L.off, a.e[id2]);
    }
    if (u.phi && t >= 0) apply_update(u, t - L.off, ev);
  }
}

// smoothing sweep of one colour at level l of every active instance with l < tail_first
template <typename T>
__device__ void phase_smooth(const Ctx<T>& c, int l, int color, int zero_init, int fuse_update) {
  const BatchArgs& A = c.A;
  const int* pre = A.pre + (1 + l) * (A.ninst + 1);
  const int total = pre[c.i_hi];
  const int R = A.rows_per_unit;
  for (int u = pre[c.i_lo] + c.gwarp; u < total; u += c.nwarps) {
    const int i = find_inst(pre, A.ninst, u);
    if (!ld_flag(A.active + i)) continue;
    const BatchInst I = ldg_struct(A.inst + i);
    const LevelDesc L = ldg_struct(A.lv + I.lv_off + l);
    const int nrc = (L.ny + R - 1) / R;
    const int q = u - pre[i];
    const int k = q / nrc, j0 = (q - k * nrc) * R;
    Upd up{nullptr, 0.0, 0, 0.0f};
    if (fuse_update) up = Upd{I.phi, I.clamp, ld_flag(&I.resid.stats->zero_phi), (float)I.clamp};
    const int hx = (L.nx + 1) >> 1;
    if constexpr (sizeof(T) == sizeof(float)) {
      // FP32: latency-bound, so the rows' loads go out together
      const PlaneCoef<T> cf = ldg_struct(c.mg.coef + L.coef_off + k);
      const int nr = min(R, L.ny - j0);
      for (int ip = c.lane; ip < hx; ip += 32) smooth_rows(c.mg, L, cf, ip, j0, nr, k, color, zero_init, up);
    } else {
      // FP64: bound by the FP64 pipe; the row-at-a-time form keeps fewer registers
      // (measured: 640 against 580 Mcell-steps/s on the 64-instance sweep)
      for (int j = j0; j < j0 + R && j < L.ny; ++j)
        for (int ip = c.lane; ip < hx; ip += 32) smooth_pair(c.mg, L, ip, j, k, color, zero_init, up);
    }
  }
}

// restriction (op 0) or prolongation (op 1) between levels l and l+1
template <typename T>
__device__ void phase_transfer(const Ctx<T>& c, int l, int op) {
  const BatchArgs& A = c.A;
  const int* pre = A.pre + (1 + A.Ldown + l) * (A.ninst + 1);
  const int total = pre[c.i_hi];
  const int R = A.rows_per_unit;
  for (int u = pre[c.i_lo] + c.gwarp; u < total; u += c.nwarps) {
    const int i = find_inst(pre, A.ninst, u);
    if (!ld_flag(A.active + i)) continue;
    const BatchInst I = ldg_struct(A.inst + i);
    const LevelDesc F = ldg_struct(A.lv + I.lv_off + l), Cc = ldg_struct(A.lv + I.lv_off + l + 1);
    const int nrc = (Cc.ny + R - 1) / R;
    const int q = u - pre[i];
    const int K = q / nrc, J0 = (q - K * nrc) * R;
    for (int J = J0; J < J0 + R && J < Cc.ny; ++J)
      for (int I0 = c.lane; I0 < Cc.nx; I0 += 32) {
        if (op == 0) restrict_cell(c.mg, F, Cc, I0, J, K, black_residual_zero(F, A.nu1));
        else prolong_cell(c.mg, F, Cc, I0, J, K, 0);
      }
  }
}

// the tail levels of every active instance: one block per instance
template <typename T>
__device__ void phase_tail(const Ctx<T>& c, unsigned char* smem) {
  const BatchArgs& A = c.A;
  for (int i = c.i_lo + c.grank; i < c.i_hi; i += c.ncta) {
    if (!ld_flag(A.active + i)) continue;
    const BatchInst I = ldg_struct(A.inst + i);
    TailArgs t{A.lvt + I.lvt_off, I.nlev_tail, I.tail_elems, I.tail_base, A.nu1, A.nu2,
               I.bottom_sweeps, 0,
               I.dense_lev >= 0 ? static_cast<const T*>(A.dense) + I.dense_off : nullptr,
               I.dense_lev, 0};
    tail_vcycle<T>(c.mg, t, smem);
  }
}

// phi += e for instances whose update is not folded into a sweep (all levels in the tail)
template <typename T>
__device__ void phase_update(const Ctx<T>& c) {
  const BatchArgs& A = c.A;
  const int* pre = A.pre;
  const int total = pre[c.i_hi];
  for (int u = pre[c.i_lo] + c.gwarp; u < total; u += c.nwarps) {
    const int i = find_inst(pre, A.ninst, u);
    const BatchInst I = ldg_struct(A.inst + i);
    if (!ld_flag(A.active + i) || I.tail_first != 0) continue;
    const int j = u - pre[i];
    const LevelDesc L = ldg_struct(A.lv + I.lv_off);
    const Upd up{I.phi, I.clamp, ld_flag(&I.resid.stats->zero_phi), (float)I.clamp};
    for (int k = 0; k < L.nz; ++k)
      for (int x = c.lane; x < L.nx; x += 32) {
        const long long id = L.off + ((long long)k * L.ny + j) * L.nx + x;
        apply_update(up, id - L.off, c.mg.e[id]);
      }
  }
}

template <typename T>
__global__ void __launch_bounds__(512, 1) batch_kernel(BatchArgs A) {
  extern __shared__ __align__(16) unsigned char bsmem[];
  MGArgs<T> mg;
  mg.e = static_cast<T*>(A.e);
  mg.r = static_cast<T*>(A.r);
  mg.s = static_cast<T*>(A.s);
  mg.coef = static_cast<const PlaneCoef<T>*>(A.coef);
  mg.lv = A.lv;
  const int lane = threadIdx.x & 31;
  // this CTA's group: its CTAs, instances and barrier
  const int g = find_inst(A.grp_cta, A.ngroups, (int)blockIdx.x);
  const int cta_lo = A.grp_cta[g], ncta = A.grp_cta[g + 1] - cta_lo;
  const int grank = (int)blockIdx.x - cta_lo;
  GridBar* gbar = A.bar + g;
  const int gwarp = (grank * (int)blockDim.x + (int)threadIdx.x) >> 5;
  const int nwarps = (ncta * (int)blockDim.x) >> 5;
  const Ctx<T> c{A, mg, lane, gwarp, nwarps, A.grp_inst[g], A.grp_inst[g + 1], grank, ncta};
  const int nsteps = A.mode == 1 ? 1 : *A.nsteps;
  int nbar = 0;
#define FX_BAR()                                                                    \
  do {                                                                              \
    ++nbar;                                                                         \
    if (!grid_barrier(gbar, A.status, (unsigned)ncta, kBarrierSpinCycles, A.dbg, nbar)) { \
      if (A.dbg && threadIdx.x == 0) A.dbg[8 + blockIdx.x] = -nbar;                 \
      return;                                                                       \
    }                                                                               \
  } while (0)
  for (int step = 0; step < nsteps; ++step) {
    // every instance of the group takes part in the step; the barrier before the
    // reset keeps it from racing with slower blocks still reading the previous
    // step's flags
    if (step > 0) FX_BAR();
    for (int i = c.i_lo + grank * (int)blockDim.x + (int)threadIdx.x; i < c.i_hi;
         i += ncta * (int)blockDim.x)
      A.active[i] = 1;
    FX_BAR();
    phase_tdgl(c, A.mode == 1 ? 3 : 0);          // Step 1a (or the RHS of the current P)
    FX_BAR();
    for (int cyc = 0;; ++cyc) {
      phase_resid(c, cyc == 0, A.mode == 0 && cyc == 0);
      FX_BAR();
      phase_decide(c, cyc == 0);
      FX_BAR();
      int any = 0;
      for (int i = c.i_lo; i < c.i_hi; ++i) any |= ld_flag(A.active + i);
      if (!any) break;
      // one V-cycle on the active instances
      for (int l = 0; l < A.Ldown; ++l) {
        for (int sw = 0; sw < A.nu1; ++sw) {
          phase_smooth(c, l, 0, sw == 0, 0);
          FX_BAR();
          phase_smooth(c, l, 1, 0, 0);
          FX_BAR();
        }
        phase_transfer(c, l, 0);
        FX_BAR();
      }
      phase_tail(c, bsmem);
      FX_BAR();
      for (int l = A.Ldown - 1; l >= 0; --l) {
        phase_transfer(c, l, 1);
        FX_BAR();
        for (int sw = 0; sw < A.nu2; ++sw) {
          phase_smooth(c, l, 0, 0, 0);
          FX_BAR();
          phase_smooth(c, l, 1, 0, l == 0 && sw == A.nu2 - 1);
          FX_BAR();
        }
      }
      if (A.any_full_tail || A.nu2 == 0) {
        phase_update(c);
        FX_BAR();
      }
    }
    if (A.mode == 0 && grank == 0)
      for (int i = c.i_lo + (int)threadIdx.x; i < c.i_hi; i += blockDim.x)
        A.inst[i].resid.stats->steps += 1;
  }
  if (A.dbg && threadIdx.x == 0) A.dbg[8 + blockIdx.x] = nbar;
#undef FX_BAR
}

// ---- the same phases as separate kernels of a CUDA graph -----------------------------
// One launch per phase over the whole grid (a single CTA group spanning every
// instance), so each phase keeps only its own registers, and kernel boundaries
// take the place of the grid barriers.  The per-cell operations and the
// per-instance sums are those of batch_kernel (the TDGL update and the
// decisions are mapped onto threads differently), so the two engines give
// identical results.

template <typename T>
__device__ __forceinline__ MGArgs<T> batch_mg(const BatchArgs& A) {
  MGArgs<T> mg;
  mg.e = static_cast<T*>(A.e);
  mg.r = static_cast<T*>(A.r);
  mg.s = static_cast<T*>(A.s);
  mg.coef = static_cast<const PlaneCoef<T>*>(A.coef);
  mg.lv = A.lv;
  return mg;
}

// warps of the whole grid share the units; CTAs are ranked for the per-instance tail
template <typename T>
__device__ __forceinline__ Ctx<T> grid_ctx(const BatchArgs& A) {
  const int gwarp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
  return Ctx<T>{A, batch_mg<T>(A), (int)(threadIdx.x & 31), gwarp, nwarps, 0, A.ninst, (int)blockIdx.x,
                (int)gridDim.x};
}

__global__ void __launch_bounds__(256) ph_activate_kernel(BatchArgs A) {
  pdl_enter();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < A.ninst; i += gridDim.x * blockDim.x)
    A.active[i] = 1;
}

// TDGL update (or right-hand side only, mode 3) of the graph engine: one block per
// 32 x 2 column tile of one instance, each column's dynamic planes split into
// kTdglChunks chunks marched by one thread each.  A chunk's first and last right-
// hand sides need the neighbouring chunks' new P, exchanged through shared memory.
// The operations per cell are tdgl_column's (force_z, advance, rhs_value on the
// same new-P values), so both engines give identical results; the persistent
// kernel keeps one thread per column (its blocks are one-dimensional).
__global__ void __launch_bounds__(kTdglTileX* kTdglTileY* kTdglChunks) ph_tdgl_chunk_kernel(BatchArgs A, int mode) {
  pdl_enter();
  __shared__ double first_s[kTdglChunks][kTdglTileY][kTdglTileX], last_s[kTdglChunks][kTdglTileY][kTdglTileX];
  const int inst = find_inst(A.tile_pre, A.ninst, (int)blockIdx.x);
  TDGLArgs a = ldg_struct(A.inst + inst).tdgl;
  a.mode = mode;
  const int tile = (int)blockIdx.x - A.tile_pre[inst];
  const int tiles_x = (a.nx + kTdglTileX - 1) / kTdglTileX;
  const int ty_tile = tile / tiles_x, tx_tile = tile - ty_tile * tiles_x;
  const int tx = threadIdx.x, ty = threadIdx.y, c = threadIdx.z;
  const int i = tx_tile * kTdglTileX + tx, j = ty_tile * kTdglTileY + ty;
  const bool col = i < a.nx && j < a.ny;
  const int per = (a.kd_hi - a.kd_lo + 1 + kTdglChunks - 1) / kTdglChunks;
  const int k0 = a.kd_lo + c * per, k1 = min(a.kd_hi, k0 + per - 1);   // empty when k0 > k1
  const long long plane = (long long)a.nx * a.ny;
  const long long cix = (long long)j * a.nx + i;
  const double v_bot = a.params->v_bot, v_top = a.params->v_top;
  double pm2 = 0.0, pm1 = 0.0, p_first = 0.0, p_second = 0.0;
  if (col && k0 <= k1) {
    const int im = (i == 0) ? a.nx - 1 : i - 1, ip = (i == a.nx - 1) ? 0 : i + 1;
    const int jm = (j == 0) ? a.ny - 1 : j - 1, jp = (j == a.ny - 1) ? 0 : j + 1;
    for (int k = k0; k <= k1; ++k) {
      const long long t = k * plane + cix;
      double pn = 0.0;
      if (__ldg(&a.planes[k].fe)) {
        if (mode == 3) {
          pn = a.P_in[t];
        } else {
          const PlaneTDGL pt = ldg_struct(a.planes + k);
          const double f = force_z(a, pt, a.planes, a.P_in, a.phi, t, k, i, j, im, ip, jm, jp, v_bot, v_top);
          pn = advance(a, t, f);
          a.P_out[t] = pn;
        }
      }
      if (k == k0) p_first = pn;
      if (k == k0 + 1) p_second = pn;
      if (k >= k0 + 2) a.b[(k - 1) * plane + cix] = rhs_value(a, a.planes, k - 1, pm2, pm1, pn, v_bot, v_top);
      pm2 = pm1;
      pm1 = pn;
    }
    first_s[c][ty][tx] = p_first;
    last_s[c][ty][tx] = pm1;
  }
  __syncthreads();
  if (!col || k0 > k1) return;
  const double below = k0 - 1 >= a.kd_lo ? last_s[c - 1][ty][tx] : 0.0;
  const double above = k1 + 1 <= a.kd_hi ? first_s[c + 1][ty][tx] : 0.0;
  if (k1 == k0) {
    a.b[k0 * plane + cix] = rhs_value(a, a.planes, k0, below, p_first, above, v_bot, v_top);
  } else {
    a.b[k0 * plane + cix] = rhs_value(a, a.planes, k0, below, p_first, p_second, v_bot, v_top);
    a.b[k1 * plane + cix] = rhs_value(a, a.planes, k1, pm2, pm1, above, v_bot, v_top);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) ph_resid_kernel(BatchArgs A, int first, int copy_back) {
  pdl_enter();
  phase_resid(grid_ctx<T>(A), first, copy_back);
}

// The per-instance decisions, one single-warp block per instance so that their
// FP64 sums and tests spread over the SMs (in one block they kept one SM's FP64
// pipe 80% busy for 43 us); the last block to finish sets WHILE = any instance
// still active.
template <typename T>
__global__ void __launch_bounds__(32) ph_decide_kernel(BatchArgs A, int first, unsigned long long handle) {
  pdl_enter();
  const Ctx<T> c{A, batch_mg<T>(A), (int)(threadIdx.x & 31), (int)blockIdx.x, (int)gridDim.x,
                 0, A.ninst, 0, 1};
  phase_decide(c, first);
  __shared__ int last;
  if (threadIdx.x == 0) {
    __threadfence();   // this block's flags before its ticket
    // wraps to 0 after the last block: exactly one block of every launch is last
    last = atomicInc(A.ticket, gridDim.x - 1) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  int mine = 0;
  for (int i = threadIdx.x; i < A.ninst; i += blockDim.x) mine |= ld_flag(A.active + i);
  const int any = __syncthreads_or(mine);
  if (threadIdx.x == 0) {
    if (A.any_out) *A.any_out = any;   // eager replay: the host drives the loop
    if (handle) cudaGraphSetConditional((cudaGraphConditionalHandle)handle, any ? 1u : 0u);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) ph_smooth_kernel(BatchArgs A, int l, int color, int zero_init,
                                                        int fuse_update) {
  pdl_enter();
  phase_smooth(grid_ctx<T>(A), l, color, zero_init, fuse_update);
}

template <typename T>
__global__ void __launch_bounds__(256) ph_transfer_kernel(BatchArgs A, int l, int op) {
  pdl_enter();
  phase_transfer(grid_ctx<T>(A), l, op);
}

template <typename T>
__global__ void __launch_bounds__(512) ph_tail_kernel(BatchArgs A) {
  extern __shared__ __align__(16) unsigned char psmem[];
  pdl_enter();
  phase_tail(grid_ctx<T>(A), psmem);
}

template <typename T>
__global__ void __launch_bounds__(256) ph_update_kernel(BatchArgs A) {
  pdl_enter();
  phase_update(grid_ctx<T>(A));
}

__global__ void ph_steps_kernel(BatchArgs A) {
  pdl_enter();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < A.ninst; i += gridDim.x * blockDim.x)
    A.inst[i].resid.stats->steps += 1;
}

// Failure-detection check: block 1 never arrives, so block 0's bounded wait
// must run out and record FERROX_ETIMEOUT.
__global__ void barrier_timeout_kernel(GridBar* gb, int* status, long long limit) {
  if (blockIdx.x == 1) return;
  grid_barrier(gb, status, gridDim.x, limit);
}

}  // namespace

cudaError_t launch_barrier_timeout(GridBar* gb, int* status, long long limit, cudaStream_t s) {
  barrier_timeout_kernel<<<2, 32, 0, s>>>(gb, status, limit);
  return cudaGetLastError();
}

template <typename T>
cudaError_t batch_prepare(size_t smem) {
  return cudaFuncSetAttribute(batch_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <typename T>
cudaError_t batch_occupancy(int threads, size_t smem, int* blocks_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, batch_kernel<T>, threads, smem);
}

template <typename T>
cudaError_t launch_batch(const BatchArgs& a, int blocks, int threads, size_t smem, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, batch_kernel<T>, a);
}

template <typename T>
cudaError_t phase_prepare(size_t tail_smem) {
  return cudaFuncSetAttribute(ph_tail_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tail_smem);
}

// One time step (mode 0) or one Poisson solve (mode 1) of every instance as a
// sequence of phase launches on the capturing stream s, the solve loop in a
// WHILE node whose body is captured on s2 (the conditional handle is created
// on the graph s is capturing into).
template <typename T>
cudaError_t capture_phases(const BatchArgs& a, int unit_blocks, size_t tail_smem, cudaStream_t s,
                           cudaStream_t s2) {
  cudaError_t e;
  const dim3 ub(unit_blocks), ut(256);
  const int mode = a.mode;
  // the decision kernels' ticket starts every graph launch at 0
  if ((e = cudaMemsetAsync(a.ticket, 0, sizeof(unsigned int), s)) != cudaSuccess) return e;
  if ((e = launch_k(ph_activate_kernel, dim3(1), dim3(256), 0, s, a)) != cudaSuccess) return e;
  if ((e = launch_k(ph_tdgl_chunk_kernel, dim3(a.ntiles), dim3(kTdglTileX, kTdglTileY, kTdglChunks), 0, s, a,
                    mode == 1 ? 3 : 0)) != cudaSuccess)
    return e;
  if ((e = launch_k(ph_resid_kernel<T>, ub, ut, 0, s, a, 1, mode == 0 ? 1 : 0)) != cudaSuccess) return e;
  cudaStreamCaptureStatus st;
  cudaGraph_t g;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  if ((e = cudaStreamGetCaptureInfo(s, &st, nullptr, &g, nullptr, nullptr, nullptr)) != cudaSuccess) return e;
  cudaGraphConditionalHandle h;
  if ((e = cudaGraphConditionalHandleCreate(&h, g, 0, 0)) != cudaSuccess) return e;
  if ((e = launch_k(ph_decide_kernel<T>, dim3(a.ninst), dim3(32), 0, s, a, 1, (unsigned long long)h)) != cudaSuccess)
    return e;
  if ((e = cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, nullptr, &nd)) != cudaSuccess) return e;
  cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cn;
  if ((e = cudaGraphAddNode(&cn, g, deps, nullptr, nd, &cp)) != cudaSuccess) return e;
  if ((e = cudaStreamBeginCaptureToGraph(s2, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                         cudaStreamCaptureModeRelaxed)) != cudaSuccess)
    return e;
  // one V-cycle on the active instances, then their residual and decisions
  for (int l = 0; l < a.Ldown; ++l) {
    for (int sw = 0; sw < a.nu1; ++sw) {
      launch_k(ph_smooth_kernel<T>, ub, ut, 0, s2, a, l, 0, sw == 0 ? 1 : 0, 0);
      launch_k(ph_smooth_kernel<T>, ub, ut, 0, s2, a, l, 1, 0, 0);
    }
    launch_k(ph_transfer_kernel<T>, ub, ut, 0, s2, a, l, 0);
  }
  launch_k(ph_tail_kernel<T>, dim3(a.ninst), dim3(512), tail_smem, s2, a);
  for (int l = a.Ldown - 1; l >= 0; --l) {
    launch_k(ph_transfer_kernel<T>, ub, ut, 0, s2, a, l, 1);
    for (int sw = 0; sw < a.nu2; ++sw) {
      launch_k(ph_smooth_kernel<T>, ub, ut, 0, s2, a, l, 0, 0, 0);
      launch_k(ph_smooth_kernel<T>, ub, ut, 0, s2, a, l, 1, 0, (l == 0 && sw == a.nu2 - 1) ? 1 : 0);
    }
  }
  if (a.any_full_tail || a.nu2 == 0) launch_k(ph_update_kernel<T>, ub, ut, 0, s2, a);
  launch_k(ph_resid_kernel<T>, ub, ut, 0, s2, a, 0, 0);
  launch_k(ph_decide_kernel<T>, dim3(a.ninst), dim3(32), 0, s2, a, 0, (unsigned long long)h);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  cudaGraph_t body_out;
  if ((e = cudaStreamEndCapture(s2, &body_out)) != cudaSuccess) return e;
  if ((e = cudaStreamUpdateCaptureDependencies(s, &cn, nullptr, 1, cudaStreamSetCaptureDependencies)) !=
      cudaSuccess)
    return e;
  if (mode == 0) launch_k(ph_steps_kernel, dim3(1), dim3(256), 0, s, a);
  return cudaGetLastError();
}

// One time step (mode 0) of every instance with the graph engine's kernels
// launched one by one on s (no graph), the solve loop driven from the host by the
// decision kernel's "any instance active" flag: the same kernels in the same
// order, so the state advances exactly as a step of the graph.  Each launch is
// bracketed by CUDA events; ms and launches accumulate per class.
template <typename T>
cudaError_t profile_phases(const BatchArgs& a0, int unit_blocks, size_t tail_smem, cudaStream_t s, int* any_dev,
                           int* any_host, int max_cycles, double* ms, int* launches) {
  enum { WAIT = -1, TDGL, RESID, DECIDE, SMOOTH_FINE, SMOOTH_COARSE, TRANSFER, TAIL, OTHER };
  BatchArgs a = a0;
  a.mode = 0;
  a.any_out = any_dev;
  const dim3 ub(unit_blocks), ut(256);
  // (class, start event); the next mark ends the interval.  WAIT intervals hold
  // the host's read of the flag (no launch): neither timed nor counted.
  std::vector<std::pair<int, cudaEvent_t>> marks;
  cudaError_t err = cudaSuccess;
  auto mark = [&](int cls) {
    cudaEvent_t e;
    if (err == cudaSuccess) err = cudaEventCreate(&e);
    if (err == cudaSuccess) err = cudaEventRecord(e, s);
    if (err == cudaSuccess) marks.push_back({cls, e});
  };
  auto note = [&](cudaError_t e) { if (err == cudaSuccess) err = e; };
  auto read_any = [&]() -> int {
    if (err == cudaSuccess) err = cudaMemcpyAsync(any_host, any_dev, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    return err == cudaSuccess ? *any_host : 0;
  };
  note(cudaMemsetAsync(a.ticket, 0, sizeof(unsigned int), s));
  mark(OTHER);
  note(launch_k(ph_activate_kernel, dim3(1), dim3(256), 0, s, a));
  mark(TDGL);
  note(launch_k(ph_tdgl_chunk_kernel, dim3(a.ntiles), dim3(kTdglTileX, kTdglTileY, kTdglChunks), 0, s, a, 0));
  mark(RESID);
  note(launch_k(ph_resid_kernel<T>, ub, ut, 0, s, a, 1, 1));
  mark(DECIDE);
  note(launch_k(ph_decide_kernel<T>, dim3(a.ninst), dim3(32), 0, s, a, 1, 0ULL));
  mark(WAIT);
  int any = read_any();
  for (int cyc = 0; any && cyc <= max_cycles; ++cyc) {
    for (int l = 0; l < a.Ldown; ++l) {
      for (int sw = 0; sw < a.nu1; ++sw) {
        mark(l == 0 ? SMOOTH_FINE : SMOOTH_COARSE);
        note(launch_k(ph_smooth_kernel<T>, ub, ut, 0, s, a, l, 0, sw == 0 ? 1 : 0, 0));
        mark(l == 0 ? SMOOTH_FINE : SMOOTH_COARSE);
        note(launch_k(ph_smooth_kernel<T>, ub, ut, 0, s, a, l, 1, 0, 0));
      }
      mark(TRANSFER);
      note(launch_k(ph_transfer_kernel<T>, ub, ut, 0, s, a, l, 0));
    }
    mark(TAIL);
    note(launch_k(ph_tail_kernel<T>, dim3(a.ninst), dim3(512), tail_smem, s, a));
    for (int l = a.Ldown - 1; l >= 0; --l) {
      mark(TRANSFER);
      note(launch_k(ph_transfer_kernel<T>, ub, ut, 0, s, a, l, 1));
      for (int sw = 0; sw < a.nu2; ++sw) {
        mark(l == 0 ? SMOOTH_FINE : SMOOTH_COARSE);
        note(launch_k(ph_smooth_kernel<T>, ub, ut, 0, s, a, l, 0, 0, 0));
        mark(l == 0 ? SMOOTH_FINE : SMOOTH_COARSE);
        note(launch_k(ph_smooth_kernel<T>, ub, ut, 0, s, a, l, 1, 0, (l == 0 && sw == a.nu2 - 1) ? 1 : 0));
      }
    }
    if (a.any_full_tail || a.nu2 == 0) {
      mark(OTHER);
      note(launch_k(ph_update_kernel<T>, ub, ut, 0, s, a));
    }
    mark(RESID);
    note(launch_k(ph_resid_kernel<T>, ub, ut, 0, s, a, 0, 0));
    mark(DECIDE);
    note(launch_k(ph_decide_kernel<T>, dim3(a.ninst), dim3(32), 0, s, a, 0, 0ULL));
    mark(WAIT);
    any = read_any();
  }
  mark(OTHER);
  note(launch_k(ph_steps_kernel, dim3(1), dim3(256), 0, s, a));
  mark(WAIT);
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  for (size_t q = 0; q + 1 < marks.size(); ++q) {
    if (marks[q].first == WAIT) continue;
    float t = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&t, marks[q].second, marks[q + 1].second);
    ms[marks[q].first] += t;
    ++launches[marks[q].first];
  }
  for (auto& m : marks) cudaEventDestroy(m.second);
  return err;
}

template cudaError_t profile_phases<double>(const BatchArgs&, int, size_t, cudaStream_t, int*, int*, int, double*, int*);
template cudaError_t profile_phases<float>(const BatchArgs&, int, size_t, cudaStream_t, int*, int*, int, double*, int*);
template cudaError_t phase_prepare<double>(size_t);
template cudaError_t phase_prepare<float>(size_t);
template cudaError_t capture_phases<double>(const BatchArgs&, int, size_t, cudaStream_t, cudaStream_t);
template cudaError_t capture_phases<float>(const BatchArgs&, int, size_t, cudaStream_t, cudaStream_t);
template cudaError_t batch_prepare<double>(size_t);
template cudaError_t batch_prepare<float>(size_t);
template cudaError_t batch_occupancy<double>(int, size_t, int*);
template cudaError_t batch_occupancy<float>(int, size_t, int*);
template cudaError_t launch_batch<double>(const BatchArgs&, int, int, size_t, cudaStream_t);
template cudaError_t launch_batch<float>(const BatchArgs&, int, int, size_t, cudaStream_t);

}  // namespace fx

// Internal declarations shared by the kernels and the host engine of libferrox.
//
// Scaled form of the Poisson problem used on the device: lengths in units of the
// fine cell size h0, permittivity in units of eps0, and every cell equation
// multiplied by h0^2/eps0.  The operator coefficients are then the relative
// permittivities (level 0), the right-hand side is b' = b h0^2/eps0, and the
// potential stays in volts.  The solution is unchanged by the scaling.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstring>

#include "../../include/ferrox.h"

#include <utility>

namespace fx {

// Programmatic dependent launch: each solver kernel is launched with the
// programmatic-serialization attribute and first waits for the kernel before
// it to complete (its memory visible).  No kernel triggers its dependents
// early: they are released when it completes, so blocks of the next kernel
// never sit on SMs waiting while this one still has blocks to place (measured:
// an early trigger cost 3% in FP64, 2% in the mixed form); what remains is the
// launch work the driver does ahead of time.  Without the attribute the wait
// is a no-op.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

int pdl_enabled();

template <typename... K, typename... A>
inline cudaError_t launch_k(void (*kern)(K...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                            A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<A>(args)...);
}

constexpr int kMaxLevels = 24;
constexpr int kTailMaxCells = 4096;     // levels at or below this size run in one CTA (FP32)
constexpr int kTailMaxCellsFP64 = 512;  // the same for FP64 corrections
constexpr int kTailThreads = 1024;
constexpr int kDenseMax = 64;           // a tail level of at most this many cells is solved by its inverse
constexpr int kDenseWide = 512;         // a first tail level up to this size (stacks without
                                        // carriers) is solved by its inverse across the SMs
                                        // instead of the tail V-cycle
constexpr int kTailMaxSmem = 200 * 1024; // shared memory available to the tail CTA
constexpr int kResidBX = 32, kResidBY = 8; // residual: one thread per (x, y) column
constexpr int kTdglTileX = 32, kTdglTileY = 2, kTdglChunks = 4;  // batched TDGL: column tile, z chunks

// Copy of a read-only table entry through the read-only data path (8-byte
// loads); fields the caller never uses are removed by the compiler.  The words
// land in an integer buffer and reach the struct by memcpy: storing them through
// an integer pointer into the struct and then reading its double or int fields
// breaks the aliasing rules, and the optimiser may then read fields it considers
// never written.
template <typename S>
__device__ __forceinline__ S ldg_struct(const S* p) {
  static_assert(sizeof(S) % 8 == 0, "table entries are padded to 8 bytes");
  unsigned long long w[sizeof(S) / 8];
  const unsigned long long* src = reinterpret_cast<const unsigned long long*>(p);
#pragma unroll
  for (int q = 0; q < (int)(sizeof(S) / 8); ++q) w[q] = __ldg(src + q);
  S out;
  memcpy(&out, w, sizeof(S));
  return out;
}

// ---- per-plane data of the fine level (device, read-only during a step) -------------
struct PlaneTDGL {
  int fe;          // ferroelectric plane
  int b_dyn;       // b may be nonzero from P on this plane (FE or FE-adjacent)
  int sc;          // semiconductor plane
  int fd;          // Fermi-Dirac carriers (else Boltzmann)
  double alpha, beta, gamma;          // z component
  double alpha_xy, beta_xy, gamma_xy; // in-plane components
  double g11, g44, Gamma;
  double wz_dn, wz_c, wz_up;          // d2/dz2 weights incl. 1/h^2 and the P-BC stencil
  // lower face (k-1/2) of the plane: face potential and face polarization weights
  double fw_L, fw_R, fpc;             // Phi_f = fw_L Phi_{k-1} + fw_R Phi_k - fpc (P_k - P_{k-1})
  double lift;                        // scaled Dirichlet lift (multiplies V of the adjacent electrode)
  double eps_r;
  // carriers (scaled): rho' = kq (p0 e^{-phi/VT} - n0 e^{phi/VT} + Nnet), s' = kq (n + p)/VT
  double kq, n0, p0, Nnet, inv_vt;
  // Fermi-Dirac: n = Nc F(eta_e0 + phi/VT), p = Nv F(eta_p0 - phi/VT)
  double Nc, Nv, eta_e0, eta_p0;
  // kq n0, kq p0, kq Nnet (the double-float residual forms rho from these)
  double kqn0, kqp0, kqN;
};

// ---- per-plane multigrid coefficients of one level ----------------------------------
template <typename T>
struct PlaneCoef {
  T cx, cy;      // lateral couplings (0 when that lateral size is 1)
  T czlo, czhi;  // couplings through the lower / upper z face (electrode faces included)
  T diag;        // 2 cx + 2 cy + czlo + czhi
  T invdiag;
  int has_s;     // semiconductor shift present on this plane
  int pad;
};

// fine-level coefficients as double-float pairs (h + l = the FP64 value to 2^-48),
// for the double-float outer residual of the mixed form
struct PlaneCoefDF {
  float cx_h, cx_l, cy_h, cy_l, czlo_h, czlo_l, czhi_h, czhi_l, diag_h, diag_l;
};

struct LevelDesc {
  int nx, ny, nz;
  int crx, cry, crz;  // this level is coarsened in x / y / z to form the next one
  long long ncell;
  long long off;      // element offset of the level inside the level arenas
  int coef_off;       // offset of the level's planes in the coefficient tables
  int pad;
};

// ---- small device-side state ---------------------------------------------------------
struct DevParams {
  double v_bot, v_top;
};

struct DevStats {
  long long steps, solves, cycles, launches;
  int last_cond, pad2;
  double bnorm2;          // ||b||^2 of the current solve (b is fixed within a solve)
  int last_cycles, status;
  double last_rel;
  double last_rnorm, last_scale;
  unsigned int done_ctr;
  int cycles_this_solve;
  int zero_phi;
  int inner_k;            // adaptive inner cycles: V-cycles of the current outer iteration
  int inner_left;         //   ... still to run
  int pad3;
  double rho_v;           //   estimated contraction per V-cycle (0: none yet), kept across solves
  double prev_rnorm;      //   ||r|| at the previous outer iteration of this solve
  long long vcycles;      // V-cycles run, all solves (inner cycles included)
  long long nn_rejected;  // learned corrections rejected (they did not lower ||r||)
};

// Arguments of the outer (FP64) residual kernel.
struct ResidArgs {
  const double* phi;
  const double* b;
  const PlaneTDGL* planes;
  const PlaneCoef<double>* coef0;
  const DevParams* params;
  int nx, ny, nz;
  void* r_out;         // float or double (level-0 residual)
  void* s_out;         // float or double (level-0 Newton shift), may be null
  double* partials;    // [3][number of residual blocks]
  DevStats* stats;
  double tol;
  int max_cycles;
  int first;           // first residual of a solve
  int set_cond;        // call cudaGraphSetConditional
  unsigned long long cond_handle;
  int launches_per_cycle;  // kernels of one outer iteration (V-cycle + update + resid); adaptive:
                           // the fixed part (update + resid)
  int no_stats;            // write r (and s) only: no norms, no decision
  int adapt_max;           // > 0: choose the next outer iteration's V-cycles (<= adapt_max)
  int launches_per_vcycle; // adaptive: kernels of one V-cycle and its countdown
  int kchunk;              // planes per z chunk of the multi-block kernel (grid.z chunks)
  int inner_fixed;         // fixed V-cycles per outer iteration (when adapt_max == 0)
  double* norm_out;        // store ||r|| here instead of taking a decision
  const double* reject_ref;          // ||r|| of the guess before a learned correction: the
  unsigned long long reject_handle;  // first residual sets this IF condition to 1 when
                                     // the corrected guess is no better (reject it)
  int carriers;                      // carrier charge: 0 none, 1 Boltzmann planes only, 2 with
                                     // Fermi-Dirac planes
  const PlaneCoefDF* coef_df;        // non-null: stencil in double-float arithmetic (FP32 pipe)
  void* sinv_out;                    // with s_out: 1 / (diag + s) of level 0 (float or double)
  int warp_rows;                     // nx is a multiple of 32: each warp holds 32 cells of a row
};

// ---- launchers (kernels.cu / tdgl.cu) ------------------------------------------------
template <typename T>
struct MGArgs {
  T* e;                     // level arena of corrections
  T* r;                     // level arena of right-hand sides
  T* s;                     // level arena of Newton shifts (null when no SC)
  const PlaneCoef<T>* coef; // all levels
  const LevelDesc* lv;      // device copy of the level table
  const T* sinv = nullptr;  // 1 / (diag + s) of the swept level, from the level's first cell
                            // (index id - L.off): sweeps multiply by it instead of dividing
                            // (null: divide)
};

// phi += e folded into the last fine-level black sweep
struct UpdateArgs {
  double* phi;
  const DevStats* stats;
  double clamp;
};

// levels handled by the single-CTA tail; offsets of lv are relative to the tail base
struct TailArgs {
  const LevelDesc* lv;  // device table of the tail levels (shared-memory offsets)
  int nlev;
  long long elems;      // elements per tail array in shared memory
  long long base;       // arena offset of the first tail level
  int nu1, nu2, bottom_sweeps, constant;
  const void* dense;    // T[n * n]: inverse of the operator of tail level dense_lev (null: none)
  int dense_lev;
  int pad;
};

// Direct FP64 form (V-cycle on phi itself): the fused fine-level residual +
// restriction + norm that takes the convergence decision
struct CheckArgs {
  double* partials;        // 2 per block of the check grid
  DevStats* stats;
  double tol;
  int max_cycles;
  int first;               // first check of a solve (sums ||b||^2)
  int set_cond;
  int launches_per_cycle;  // kernels of one loop iteration (one V-cycle)
  unsigned long long cond_handle;
  int first_launches;      // kernels before the first check (pre-smoothing + the check)
  int pad;
};

template <typename T>
void launch_smooth(const MGArgs<T>& a, const LevelDesc& L, int color, int zero_init,
                   const UpdateArgs* upd, cudaStream_t s, const DevStats* zero_stats = nullptr);
// fused red-black sweep (both colours in one launch, e_in -> e_out, level-relative
// arrays): smooth_rb_tile is 0 where the level cannot take it
template <typename T>
int smooth_rb_tile(const LevelDesc& L, bool has_s);
template <typename T>
cudaError_t smooth_rb_prepare();
// direct FP64 form, fine level: a colour sweep on bs = b / diag with coefficients
// divided by the diagonal (six FP64 operations per cell), and bs from b
void launch_smooth_scaled(const MGArgs<double>& a, const LevelDesc& L, int color, cudaStream_t s,
                          const DevStats* zero_stats);
void launch_scale_rhs(const double* b, const PlaneCoef<double>* coef, int nx, int ny, int nz, double* bs,
                      cudaStream_t s);
template <typename T>
void launch_smooth_rb(const MGArgs<T>& a, const LevelDesc& L, const T* e_in, T* e_out,
                      int zero_init, const UpdateArgs* upd, cudaStream_t s);
dim3 check_grid(const LevelDesc& C);
void launch_restrict_check(const MGArgs<double>& fa, double* rc, const LevelDesc& F,
                           const LevelDesc& C, int nu1, const CheckArgs& ck, cudaStream_t s);
template <typename T>
void launch_restrict(const MGArgs<T>& a, const LevelDesc& F, const LevelDesc& C, int nu1,
                     cudaStream_t s);
template <typename T>
void launch_prolong(const MGArgs<T>& a, const LevelDesc& F, const LevelDesc& C, int constant,
                    cudaStream_t s, bool tiled = false, T* fine = nullptr);
template <typename T>
size_t tail_smem_bytes(long long elems, bool has_s);
template <typename T>
cudaError_t tail_prepare(size_t smem);
template <typename T>
void launch_tail(const MGArgs<T>& a, const TailArgs& t, size_t smem, cudaStream_t s);
// e = inv r for one level (n x n dense inverse, one warp per row)
template <typename T>
void launch_dense_solve(const T* inv, int n, const T* r, T* e, cudaStream_t s);
template <typename T>
void launch_resid(const ResidArgs& a, cudaStream_t s);
template <typename T>
void launch_update(double* phi, const T* e0, long long n, const DevStats* stats, double clamp,
                   cudaStream_t s, T* zero_e = nullptr);
// adaptive inner loop: arm its condition from inner_left (first node of an outer
// iteration), and count one V-cycle down after each
void launch_inner_arm(const DevStats* st, unsigned long long handle, cudaStream_t s);
void launch_inner_countdown(DevStats* st, unsigned long long handle, cudaStream_t s);

// Per-plane coefficients of the FP32-arithmetic TDGL update (mixed form): the
// force's coefficients as floats, and the right-hand side folded into three FP64
// weights of the new P below, at and above the plane.
struct PlaneF32 {
  int fe, pad;
  float alpha, beta, gamma, g11, g44, Gamma;
  float wz_dn, wz_up, wz_sum;   // d2z = wz_dn (P_dn - P) + wz_up (P_up - P) + wz_sum P
  float fw_L, fw_R, fpc;        // lower face (k - 1/2), as in PlaneTDGL
  double c_dn, c_0, c_up;       // b = c_dn P_{k-1} + c_0 P_k + c_up P_{k+1} (+ electrode lift)
};

struct TDGLArgs {
  const double* P_in;     // [ncomp][nz][ny][nx]
  double* P_out;          // new P (FE planes written)
  const double* P_base;   // order-2 corrector: P^n (null for the predictor)
  double* F_store;        // predictor of order 2: f(P^n) written here; corrector: read
  const double* phi;
  double* b;              // scaled RHS, dynamic planes written
  const PlaneTDGL* planes;
  const DevParams* params;
  int nx, ny, nz, ncomp;
  int kd_lo, kd_hi;       // dynamic plane range
  double dt, inv_h, inv_h2, b_scale;  // b_scale = h0/eps0
  int mode;               // 0: order-1 update, 1: order-2 predictor, 2: order-2 corrector,
                          // 3: right-hand side of the current P only
  const PlaneF32* planes_f32;   // non-null: force in FP32 arithmetic (one component only)
  float dtf, inv_hf, inv_h2f;
};
void launch_tdgl(const TDGLArgs& a, cudaStream_t s);
// a single-thread kernel that spins for `cycles` SM clock cycles (bounded)
void launch_delay(long long cycles, cudaStream_t s);

struct ChargeArgs {
  const double* phi;
  const double* P;        // z component plane data (P + (ncomp-1) N)
  const PlaneTDGL* planes;
  const DevParams* params;
  int nx, ny, nz, k_int;  // k_int: lowest FE plane (interface = its lower face)
  double h, eps0;
  double eps_top, eps_bot, eps_L, eps_R;
  double* out;            // 5 doubles: sum F_int, sum Phi_f_int, sum F_top, sum F_bot
  double* partials;
};
void launch_charge(const ChargeArgs& a, cudaStream_t s);

// ---- learned warm-start network (nn.cu) -----------------------------------------------
struct NNGrid {
  int D, H, W;
};
}  // namespace fx
#include <cuda_bf16.h>
#include <string>
#include <vector>
#include <algorithm>
struct ferrox_nn;
namespace fx {
// returns true when the tensor-memory (tcgen05) kernel ran, false for the mma.sync kernel
// (f_ch0: out_f receives output channel 0 only, one float per voxel)
bool nn_conv_fwd(const __nv_bfloat16* in, int cin, const __nv_bfloat16* wk, const __nv_bfloat16* wt,
                 const float* bias, int cout, NNGrid g, int relu, __nv_bfloat16* out_bf, float* out_f,
                 int f_ch0, int* fault, cudaStream_t s);
bool nn_conv_upcat_tc(const __nv_bfloat16* a4, const __nv_bfloat16* s1, const __nv_bfloat16* wt,
                      const float* bias, NNGrid g, int relu, __nv_bfloat16* out_bf, int* fault, cudaStream_t s);
bool nn_conv_uses_tc(int cin, int cout, NNGrid g);
cudaError_t nn_tc_setup();
void nn_conv_wgrad(const __nv_bfloat16* in, int cin, const __nv_bfloat16* dout, int cout, NNGrid g,
                   float* gw, float* gb, cudaStream_t s);
void nn_pool2(const __nv_bfloat16* in, NNGrid f, int C, __nv_bfloat16* out, cudaStream_t s);
void nn_upcat(const __nv_bfloat16* a4, const __nv_bfloat16* s1, NNGrid f, __nv_bfloat16* cat, cudaStream_t s);
void nn_mask(const float* d, const __nv_bfloat16* act, long long n, __nv_bfloat16* out, cudaStream_t s);
void nn_up_grad(const float* dcat, const __nv_bfloat16* a4, NNGrid f, __nv_bfloat16* out, cudaStream_t s);
void nn_skip_grad(const float* dcat, const float* dp, const __nv_bfloat16* s1, NNGrid f,
                  __nv_bfloat16* out, cudaStream_t s);
void nn_mse(const float* y, const float* tgt, int M, __nv_bfloat16* dy, float* loss, cudaStream_t s);
void nn_adam(float* p, float* g, float* m, float* v, int n, float lr, int step, cudaStream_t s);
void nn_pack(const float* w, int cin, int cout, __nv_bfloat16* wk, __nv_bfloat16* wb, __nv_bfloat16* wkt,
             __nv_bfloat16* wbt, cudaStream_t s);
__nv_bfloat16* nn_input(ferrox_nn* N);
const float* nn_output(ferrox_nn* N);
void nn_run_forward(ferrox_nn* N, cudaStream_t s);
NNGrid nn_grid(const ferrox_nn* N);
int nn_capacity(const ferrox_nn* N);
__nv_bfloat16* nn_snap_x(ferrox_nn* N);
float* nn_snap_t(ferrox_nn* N);
void nn_note_snapshots(ferrox_nn* N, int added);
int nn_next_slot(const ferrox_nn* N);
template <typename T>
void nn_bridge_restrict(T* arena, const std::vector<LevelDesc>& lv, int to, cudaStream_t s);
template <typename T>
void nn_bridge_scale(const T* arena, const LevelDesc& L, double* scale, cudaStream_t s);
template <typename T>
void nn_bridge_features(const T* r, const LevelDesc& L, const float* pf, const double* scale,
                        const DevParams* prm, __nv_bfloat16* x, cudaStream_t s);
template <typename T>
void nn_bridge_apply(const float* y, const LevelDesc& L, const double* scale, T* e, cudaStream_t s);
template <typename T>
void nn_bridge_guess_error(const double* phi, const double* guess, long long n, T* e0, cudaStream_t s);
template <typename T>
void nn_bridge_target(const T* e, const LevelDesc& L, const double* scale, float* tgt, cudaStream_t s);

// ---- persistent batched engine (persistent.cu) ---------------------------------------
constexpr long long kBarrierSpinCycles = 2000000000LL;  // ~1 s at 2 GHz: a wait never hangs

struct GridBar {
  unsigned int count, gen, abort, pad;
};

struct BatchInst {
  TDGLArgs tdgl;        // P_in = P, P_out = Pbuf, instance arenas
  ResidArgs resid;      // r_out/s_out: the instance's level 0; stats: the instance's
  double* P;
  double* Pbuf;
  double* phi;
  double clamp;
  int fe_lo, fe_hi;
  int lv_off, nlev, tail_first, lvt_off, nlev_tail, bottom_sweeps;
  long long tail_elems, tail_base;
  long long dense_off;  // element offset of the instance's tail inverse in BatchArgs::dense
  int dense_lev;        // tail level solved by that inverse (-1: relaxed bottom level)
  int pad2;
};

struct BatchArgs {
  const BatchInst* inst;
  int ninst;
  int mode;             // 0: time steps, 1: Poisson solve only (Step 0)
  const int* nsteps;    // device: steps per launch
  void* e;              // correction arena (T)
  void* r;              // right-hand-side arena (T)
  void* s;              // Newton shift arena (T) or null
  const void* coef;     // PlaneCoef<T> of all levels of all instances
  const LevelDesc* lv;  // levels of all instances (arena offsets)
  const LevelDesc* lvt; // tail levels of all instances (shared-memory offsets)
  const void* dense;    // T: inverses of the instances' dense tail levels
  const int* pre;       // unit prefix tables: rows, smoothing rows per level, coarse rows per level
  const int* tile_pre;  // graph engine's TDGL: prefix of 32 x 2 column tiles per instance
  int ntiles;           // ... and their total
  int Ldown;            // deepest multi-block level count over instances
  double* partials;     // 3 per row unit
  int* active;          // per instance
  GridBar* bar;         // one barrier per CTA group
  const int* grp_cta;   // CTA groups: group g owns CTAs [grp_cta[g], grp_cta[g+1]) ...
  const int* grp_inst;  // ... and instances [grp_inst[g], grp_inst[g+1]); one group: the grid
  int ngroups;
  int pad3;
  int* status;          // global status (barrier time-out)
  double tol;
  int max_cycles, nu1, nu2, rows_per_unit, any_full_tail, pad;
  int* dbg;             // optional self-check record (null: off)
  unsigned int* ticket; // graph engine: blocks of the decision kernel done (0 between launches)
  int* any_out;         // eager phase replay: "any instance active" after each decision (else null)
};

cudaError_t launch_barrier_timeout(GridBar* gb, int* status, long long limit, cudaStream_t s);
cudaError_t launch_carrier_exp(const double* u, double* ep, double* em, long long n, cudaStream_t s);
cudaError_t launch_carrier_exp_df(const float* u_hl, double* ep, double* em, long long n, cudaStream_t s);
template <typename T>
cudaError_t batch_prepare(size_t smem);
template <typename T>
cudaError_t batch_occupancy(int threads, size_t smem, int* blocks_per_sm);
template <typename T>
cudaError_t launch_batch(const BatchArgs& a, int blocks, int threads, size_t smem, cudaStream_t s);
// the batched step as a graph of per-phase launches (same results as batch_kernel)
template <typename T>
cudaError_t phase_prepare(size_t tail_smem);
template <typename T>
cudaError_t capture_phases(const BatchArgs& a, int unit_blocks, size_t tail_smem, cudaStream_t s,
                           cudaStream_t s2);
// the same phases launched one by one, the solve loop driven from the host, each
// launch timed by CUDA events into ms[kPhaseClasses] / launches[kPhaseClasses]
constexpr int kPhaseClasses = 8;   // tdgl, resid, decide, fine sweeps, coarse sweeps, transfers, tail, other
template <typename T>
cudaError_t profile_phases(const BatchArgs& a, int unit_blocks, size_t tail_smem, cudaStream_t s, int* any_dev,
                           int* any_host, int max_cycles, double* ms, int* launches);
void launch_set_params(DevParams* p, double v_bot, double v_top, cudaStream_t s);
void launch_static_b(double* b, const PlaneTDGL* planes, const DevParams* prm, int nx, int ny,
                     int nz, cudaStream_t s);
void launch_extrapolate(double* phi, double* prev, long long n, cudaStream_t s);
void launch_stats_step(DevStats* st, int nsteps, int launches, cudaStream_t s);

}  // namespace fx

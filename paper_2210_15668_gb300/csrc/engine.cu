// Host engine and C ABI of libferrox (see include/ferrox.h).
//
// A context owns, for one device stack on one GPU:
//   * the per-plane material table of the fine grid (Fig. 1a stack, Table 1),
//     with the TDGL z-stencil weights that encode the P boundary conditions,
//     the flux-continuous face weights, the Dirichlet lift and the carrier data;
//   * the multigrid hierarchy: level shapes (full coarsening, or semi-coarsening
//     once a direction can no longer halve to an even size), per-plane couplings
//     of every level from the fine permittivity profile (series resistance
//     through z, parallel average across x/y), and the level arenas;
//   * CUDA graphs of the TDGL update, the Poisson solve and the whole time step.
//     The solve is a graph WHILE node whose condition the FP64 residual kernel
//     sets on the device, so a step runs to the tolerance with no host round trip.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <mutex>
#include <string>
#include <vector>

#include "ferrox_internal.cuh"

using namespace fx;

namespace {

constexpr double kEps0 = 8.8541878128e-12;
constexpr double kQ = 1.602176634e-19;
constexpr double kKB = 1.380649e-23;

std::string g_init_error;

// programmatic dependent launch on (1) unless graph capture rejected it (0)
int g_pdl = 1;

}  // namespace

int fx::pdl_enabled() { return g_pdl; }

struct ferrox_ctx {
  // geometry and numerics
  int nx = 0, ny = 0, nz = 0, ncomp = 1, pbc = 0;
  double h = 0.0, lambda = 0.0;
  std::vector<ferrox_layer> layers;
  ferrox_numerics num{};
  bool has_sc = false;
  bool shift = false;   // Newton shift in the multigrid operator (carriers, damped Newton)
  int kd_lo = 0, kd_hi = 0, fe_lo = 0, fe_hi = 0, k_int = 0;
  std::vector<double> epsr;  // per fine plane
  std::vector<PlaneTDGL> planes;
  // multigrid
  std::vector<LevelDesc> lv;
  int tail_first = 0;
  long long arena = 0;
  std::vector<LevelDesc> lv_tail;   // tail levels with shared-memory offsets
  long long tail_elems = 0;
  size_t tail_smem = 0;
  int resid_blocks = 0;
  int resid_kchunk = 0;   // planes per z chunk of the residual kernel
  int resid_kchunk_df = 0;  // the same for its double-float form (longer columns per thread)
  bool direct = false;    // FP64 V-cycles on phi itself (see direct_form)
  int dense_lev = -1;     // tail level solved by its inverse (-1: none)
  void* dense_d = nullptr;
  void* dense_wide_d = nullptr;   // FP64: inverse of the first tail level, solved instead of the tail
  int check_blocks = 0;   // blocks of the direct form's fused residual + restriction + norm
  // device memory
  cudaStream_t stream = nullptr;
  cudaStream_t cap1 = nullptr, cap2 = nullptr, cap3 = nullptr;
  double* P = nullptr;
  double* phi = nullptr;
  double* b = nullptr;
  double* Pbuf = nullptr;
  double* Fbuf = nullptr;
  double* phi_prev = nullptr;         // previous step's potential (guess = 1)
  void* e_arena = nullptr;
  void* e_alt = nullptr;              // second error array of the fused sweeps (largest such level)
  void* r_arena = nullptr;
  void* s_arena = nullptr;
  void* coef = nullptr;               // PlaneCoef<T> of all levels
  PlaneCoef<double>* coef0 = nullptr; // level 0 in FP64 (outer residual)
  PlaneCoef<double>* coef0s = nullptr; // level 0 divided by the diagonal (direct form's sweeps)
  double* bs = nullptr;                // b / diag (direct form's fine sweeps)
  void* sinv0 = nullptr;               // 1 / (diag + s) on level 0 (T; with a Newton shift)
  PlaneCoefDF* coef_df = nullptr;     // level 0 as double-float pairs (double-float residual)
  bool df_resid = false;              // the mixed form's outer residual in double-float
  PlaneTDGL* planes_d = nullptr;
  PlaneF32* planes_f32_d = nullptr;   // FP32 TDGL arithmetic only
  LevelDesc* lv_d = nullptr;
  LevelDesc* lvt_d = nullptr;
  DevParams* params_d = nullptr;
  DevStats* stats_d = nullptr;
  double* partials_d = nullptr;
  double* charge_d = nullptr;
  double* charge_part_d = nullptr;
  double* host_pinned = nullptr;      // small pinned staging for charge/stats reads
  // graphs
  cudaGraph_t gr_step = nullptr, gr_solve = nullptr, gr_tdgl = nullptr;
  cudaGraphExec_t ge_step = nullptr, ge_solve = nullptr, ge_tdgl = nullptr;
  double v_bot = 0.0, v_top = 0.0;
  // learned warm start
  ferrox_nn* nn = nullptr;
  int nn_mode = 0;                 // 0 off, 1 collect snapshots, 2 use before each solve
  int nn_level = 2;
  double* nn_scale = nullptr;
  double* phi_guess = nullptr;
  float* nn_pf = nullptr;          // per-plane features of the network level
  DevStats* nn_stats = nullptr;    // zeroed status for the prediction update
  cudaGraph_t gr_step_nn = nullptr;
  cudaGraphExec_t ge_step_nn = nullptr;
  std::string err;
};

namespace {

ferrox_status fail(ferrox_ctx* c, ferrox_status s, const std::string& msg) {
  if (c) c->err = msg; else g_init_error = msg;
  return s;
}

#define FX_CK(call)                                                                          \
  do {                                                                                       \
    cudaError_t _e = (call);                                                                 \
    if (_e != cudaSuccess)                                                                   \
      return fail(ctx, FERROX_ECUDA, std::string(#call) + ": " + cudaGetErrorString(_e));    \
  } while (0)

bool lateral_can_halve(int n) { return n % 2 == 0 && (n / 2 == 1 || (n / 2) % 2 == 0); }

// series resistance  int dz / eps_r(z)  between fine-grid coordinates z1 < z2 (units of h0)
double resistance(const std::vector<double>& epsr, double z1, double z2) {
  double R = 0.0;
  const int n = (int)epsr.size();
  for (int i = std::max(0, (int)std::floor(z1)); i < n && i < (int)std::ceil(z2); ++i) {
    const double lo = std::max(z1, (double)i), hi = std::min(z2, (double)i + 1.0);
    if (hi > lo) R += (hi - lo) / epsr[i];
  }
  return R;
}

void build_levels(ferrox_ctx* c) {
  c->lv.clear();
  LevelDesc L{};
  L.nx = c->nx; L.ny = c->ny; L.nz = c->nz;
  L.ncell = (long long)L.nx * L.ny * L.nz;
  c->lv.push_back(L);
  while ((int)c->lv.size() < kMaxLevels) {
    LevelDesc& F = c->lv.back();
    if (F.ncell <= 1) break;
    F.crx = lateral_can_halve(F.nx);
    F.cry = lateral_can_halve(F.ny);
    F.crz = (F.nz % 2 == 0);
    if (!F.crx && !F.cry && !F.crz) break;
    LevelDesc C{};
    C.nx = F.crx ? F.nx / 2 : F.nx;
    C.ny = F.cry ? F.ny / 2 : F.ny;
    C.nz = F.crz ? F.nz / 2 : F.nz;
    C.ncell = (long long)C.nx * C.ny * C.nz;
    c->lv.push_back(C);
  }
  c->lv.back().crx = c->lv.back().cry = c->lv.back().crz = 0;
  long long off = 0;
  int coff = 0;
  for (auto& l : c->lv) {
    l.off = off;
    l.coef_off = coff;
    off += (l.ncell + 31) / 32 * 32;   // keep every level 256-byte aligned
    coff += l.nz;
  }
  c->arena = off;
}

// first level of the single-CTA tail: small enough in cells and in shared memory
// wide: the context solves a first tail level of 65..kDenseWide cells by its
// inverse across the SMs (no carriers), so its tail may start there
void plan_tail(ferrox_ctx* c, size_t elem_size, bool wide = false) {
  const int L = (int)c->lv.size() - 1;
  const int narr = c->shift ? 3 : 2;
  c->tail_first = L;
  // one SM runs FP64 at 2 DFMA/clk, so in FP64 the tail starts at a smaller level;
  // with the wide dense solve the FP32 form starts there too
  const long long max_cells = (elem_size == sizeof(double) || (wide && !c->shift))
                                  ? kTailMaxCellsFP64 : kTailMaxCells;
  for (int l = 0; l <= L; ++l) {
    const long long elems = c->arena - c->lv[l].off;
    if (c->lv[l].ncell <= max_cells && (size_t)elems * elem_size * narr <= (size_t)kTailMaxSmem) {
      c->tail_first = l;
      break;
    }
  }
  const long long base = c->lv[c->tail_first].off;
  c->lv_tail.assign(c->lv.begin() + c->tail_first, c->lv.end());
  for (auto& t : c->lv_tail) t.off -= base;
  c->tail_elems = c->arena - base;
  c->tail_smem = (size_t)c->tail_elems * elem_size * narr;
  if (c->num.bottom_sweeps == 0) {     // enough sweeps to solve the coarsest level
    const LevelDesc& B = c->lv.back();
    // one cell: a single update is the exact solve (more sweeps repeat it)
    c->num.bottom_sweeps = B.ncell == 1 ? 1 : std::min(64, 2 * (B.nx + B.ny + B.nz));
  }
}

// The first tail level of at most kDenseMax cells (and more than one) is solved
// exactly by its inverse in stacks without carriers (no Newton shift on the
// diagonal, so the operator is fixed for the context's lifetime).
int dense_level(const ferrox_ctx* c) {
  if (c->shift) return -1;
  for (size_t l = 0; l < c->lv_tail.size(); ++l)
    if (c->lv_tail[l].ncell <= kDenseMax) return c->lv_tail[l].ncell > 1 ? (int)l : -1;
  return -1;
}

// Inverse of the level operator (diag - couplings, periodic in x and y, the
// electrode couplings on the diagonal) as the smoother sees it, from the
// precision-T coefficients; Gauss-Jordan elimination with partial pivoting in
// FP64, rounded to T.
template <typename T>
std::vector<T> dense_inverse(const std::vector<PlaneCoef<T>>& coef, const LevelDesc& L) {
  const int n = (int)L.ncell;
  std::vector<double> A((size_t)n * n, 0.0), X((size_t)n * n, 0.0);
  auto id = [&](int i, int j, int k) { return (k * L.ny + j) * L.nx + i; };
  for (int k = 0; k < L.nz; ++k)
    for (int j = 0; j < L.ny; ++j)
      for (int i = 0; i < L.nx; ++i) {
        const PlaneCoef<T>& p = coef[L.coef_off + k];
        double* row = &A[(size_t)id(i, j, k) * n];
        row[id(i, j, k)] += (double)p.diag;
        if (L.nx > 1) {
          row[id((i + L.nx - 1) % L.nx, j, k)] -= (double)p.cx;
          row[id((i + 1) % L.nx, j, k)] -= (double)p.cx;
        }
        if (L.ny > 1) {
          row[id(i, (j + L.ny - 1) % L.ny, k)] -= (double)p.cy;
          row[id(i, (j + 1) % L.ny, k)] -= (double)p.cy;
        }
        if (k > 0) row[id(i, j, k - 1)] -= (double)p.czlo;
        if (k < L.nz - 1) row[id(i, j, k + 1)] -= (double)p.czhi;
      }
  for (int q = 0; q < n; ++q) X[(size_t)q * n + q] = 1.0;
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(A[(size_t)r * n + col]) > std::fabs(A[(size_t)piv * n + col])) piv = r;
    if (piv != col)
      for (int q = 0; q < n; ++q) {
        std::swap(A[(size_t)piv * n + q], A[(size_t)col * n + q]);
        std::swap(X[(size_t)piv * n + q], X[(size_t)col * n + q]);
      }
    const double d = A[(size_t)col * n + col];
    for (int q = 0; q < n; ++q) { A[(size_t)col * n + q] /= d; X[(size_t)col * n + q] /= d; }
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      const double f = A[(size_t)r * n + col];
      if (f == 0.0) continue;
      for (int q = 0; q < n; ++q) {
        A[(size_t)r * n + q] -= f * A[(size_t)col * n + q];
        X[(size_t)r * n + q] -= f * X[(size_t)col * n + q];
      }
    }
  }
  return std::vector<T>(X.begin(), X.end());
}

template <typename T>
std::vector<PlaneCoef<T>> level_coefficients(const ferrox_ctx* c) {
  std::vector<PlaneCoef<T>> out;
  int fx = 1, fy = 1, fz = 1;
  for (size_t l = 0; l < c->lv.size(); ++l) {
    const LevelDesc& L = c->lv[l];
    for (int K = 0; K < L.nz; ++K) {
      double lat = 0.0;
      int has_s = 0;
      for (int i = K * fz; i < (K + 1) * fz; ++i) {
        lat += c->epsr[i];
        if (c->shift && c->planes[i].sc) has_s = 1;
      }
      lat /= fz;
      const double cx = L.nx > 1 ? lat / (double(fx) * fx) : 0.0;
      const double cy = L.ny > 1 ? lat / (double(fy) * fy) : 0.0;
      const double zlo = (K == 0) ? 0.0 : (K - 0.5) * fz;
      const double zlo_end = (K == 0) ? 0.5 * fz : (K + 0.5) * fz;
      const double czlo = 1.0 / (resistance(c->epsr, zlo, zlo_end) * fz);
      const double zhi = (K + 0.5) * fz;
      const double zhi_end = (K == L.nz - 1) ? (double)L.nz * fz : (K + 1.5) * fz;
      const double czhi = 1.0 / (resistance(c->epsr, zhi, zhi_end) * fz);
      PlaneCoef<T> pc{};
      const double diag = 2.0 * cx + 2.0 * cy + czlo + czhi;
      pc.cx = (T)cx; pc.cy = (T)cy; pc.czlo = (T)czlo; pc.czhi = (T)czhi;
      pc.diag = (T)diag; pc.invdiag = (T)(1.0 / diag); pc.has_s = has_s;
      out.push_back(pc);
    }
    if (L.crx) fx *= 2;
    if (L.cry) fy *= 2;
    if (L.crz) fz *= 2;
  }
  return out;
}

// Fermi-Dirac integral of order 1/2, normalised to e^eta for eta -> -inf, by the
// approximation of Bednarczyk & Bednarczyk (Phys. Lett. A 64, 409 (1978)) that the
// paper uses: F = 1/(e^-eta + xi), xi = (3 sqrt(pi)/4) v^(-3/8),
// v = eta^4 + 50 + 33.6 eta (1 - 0.68 e^(-0.17 (eta + 1)^2)).
double fd_half_host(double eta) {
  const double w = 1.0 - 0.68 * std::exp(-0.17 * (eta + 1.0) * (eta + 1.0));
  const double v = eta * eta * eta * eta + 50.0 + 33.6 * eta * w;
  const double xi = 0.75 * std::sqrt(M_PI) * std::pow(v, -0.375);
  return 1.0 / (std::exp(-eta) + xi);
}

// effective density of states 2 (2 pi m* k_B T / h^2)^(3/2), m* = m_rel m_e
double effective_dos(double m_rel, double T) {
  constexpr double kH = 6.62607015e-34, kME = 9.1093837015e-31;
  return 2.0 * std::pow(2.0 * M_PI * m_rel * kME * kKB * T / (kH * kH), 1.5);
}

// reduced band-edge distances at Phi = 0 that make the bulk neutral:
// Nv F(eta_p0) - Nc F(eta_e0) + N_D - N_A = 0 with eta_e0 + eta_p0 = -E_g/(k_B T)
void fd_reference(double Nc, double Nv, double Eg_eV, double T, double N_A, double N_D,
                  double* eta_e0, double* eta_p0) {
  const double gap = Eg_eV * kQ / (kKB * T);
  double lo = -gap - 60.0, hi = 60.0;   // the net charge falls with eta_e0
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    const double net = Nv * fd_half_host(-gap - mid) - Nc * fd_half_host(mid) + N_D - N_A;
    if (net > 0.0) lo = mid; else hi = mid;
  }
  *eta_e0 = 0.5 * (lo + hi);
  *eta_p0 = -gap - *eta_e0;
}

ferrox_status build_planes(ferrox_ctx* c) {
  const int nz = c->nz;
  c->planes.assign(nz, PlaneTDGL{});
  c->epsr.assign(nz, 0.0);
  std::vector<const ferrox_layer*> of(nz);
  int k = 0;
  for (const auto& L : c->layers)
    for (int q = 0; q < L.ncells; ++q) of[k++] = &L;
  const double h = c->h;
  double kappa;  // P_b = kappa (9 P0 - P1)
  if (c->pbc == FERROX_PBC_FREE) kappa = 1.0 / 8.0;
  else if (c->pbc == FERROX_PBC_ZERO) kappa = 0.0;
  else kappa = c->lambda / (3.0 * h + 8.0 * c->lambda);
  c->fe_lo = nz; c->fe_hi = -1;
  for (int z = 0; z < nz; ++z) {
    const ferrox_layer& L = *of[z];
    PlaneTDGL& p = c->planes[z];
    c->epsr[z] = L.eps_r;
    p.eps_r = L.eps_r;
    p.fe = L.kind == FERROX_FE;
    p.sc = L.kind == FERROX_SC;
    if (p.fe) {
      p.alpha = L.alpha; p.beta = L.beta; p.gamma = L.gamma;
      p.alpha_xy = L.alpha_xy; p.beta_xy = L.beta_xy; p.gamma_xy = L.gamma_xy;
      p.g11 = L.g11; p.g44 = L.g44; p.Gamma = L.Gamma;
      c->fe_lo = std::min(c->fe_lo, z);
      c->fe_hi = std::max(c->fe_hi, z);
    }
    if (p.sc) {
      const double N = L.N_D - L.N_A;
      const double root = std::sqrt(0.25 * N * N + L.n_i * L.n_i);
      double n0, p0;
      if (N <= 0) { p0 = -0.5 * N + root; n0 = p0 > 0 ? L.n_i * L.n_i / p0 : 0.0; }
      else { n0 = 0.5 * N + root; p0 = L.n_i * L.n_i / n0; }
      p.n0 = n0; p.p0 = p0; p.Nnet = N;
      p.kq = kQ * h * h / kEps0;
      p.inv_vt = kQ / (kKB * L.T);
      p.kqn0 = p.kq * n0; p.kqp0 = p.kq * p0; p.kqN = p.kq * N;
      p.fd = L.stats == FERROX_FERMI_DIRAC;
      if (p.fd) {
        p.Nc = effective_dos(L.m_e, L.T);
        p.Nv = effective_dos(L.m_p, L.T);
        fd_reference(p.Nc, p.Nv, L.E_g, L.T, L.N_A, L.N_D, &p.eta_e0, &p.eta_p0);
      }
      c->has_sc = true;
    }
  }
  for (int z = 0; z < nz; ++z) {
    PlaneTDGL& p = c->planes[z];
    const bool dn = z > 0 && c->planes[z - 1].fe, up = z < nz - 1 && c->planes[z + 1].fe;
    p.b_dyn = p.fe || dn || up;
    if (p.fe) {
      const double ih2 = 1.0 / (h * h);
      if (dn && up) {
        p.wz_dn = ih2; p.wz_c = -2.0 * ih2; p.wz_up = ih2;
      } else if (up || dn) {
        const double wn = 4.0 * (1.0 - 2.0 * kappa) / 3.0 * ih2;
        const double wc = 4.0 * (18.0 * kappa - 3.0) / 3.0 * ih2;
        p.wz_c = wc;
        p.wz_up = up ? wn : 0.0;
        p.wz_dn = dn ? wn : 0.0;
      } else {
        return fail(nullptr, FERROX_EINVAL, "a ferroelectric layer must be at least 2 cells thick");
      }
    }
    if (z > 0) {
      const double eL = c->epsr[z - 1], eR = c->epsr[z];
      p.fw_L = eL / (eL + eR);
      p.fw_R = eR / (eL + eR);
      p.fpc = h / (2.0 * kEps0 * (eL + eR));
    }
    p.lift = (z == 0 || z == nz - 1) ? 2.0 * c->epsr[z] : 0.0;
  }
  c->kd_lo = std::max(0, c->fe_lo - 1);
  c->kd_hi = std::min(nz - 1, c->fe_hi + 1);
  c->k_int = c->fe_lo;
  return FERROX_OK;
}

// ---- enqueue helpers (used while capturing) ---------------------------------------------

template <typename T>
MGArgs<T> mg_args(ferrox_ctx* c) {
  MGArgs<T> a;
  a.e = static_cast<T*>(c->e_arena);
  a.r = static_cast<T*>(c->r_arena);
  a.s = static_cast<T*>(c->s_arena);
  a.coef = static_cast<const PlaneCoef<T>*>(c->coef);
  a.lv = c->lv_d;
  return a;
}

// damped Newton in semiconductor stacks: at most 10 V_T per update
double update_clamp(const ferrox_ctx* c) {
  if (!c->has_sc) return INFINITY;
  double tmax = 0.0;
  for (const auto& L : c->layers) if (L.kind == FERROX_SC) tmax = std::max(tmax, L.T);
  return 10.0 * kKB * tmax / kQ;
}

// a plane's FP64 coefficients as double-float pairs: h = the nearest float, l = the
// nearest float to the remainder
PlaneCoefDF split_coef_df(const PlaneCoef<double>& q) {
  auto split = [](double x, float& h, float& l) {
    h = (float)x;
    l = (float)(x - (double)h);
  };
  PlaneCoefDF d;
  split(q.cx, d.cx_h, d.cx_l);
  split(q.cy, d.cy_h, d.cy_l);
  split(q.czlo, d.czlo_h, d.czlo_l);
  split(q.czhi, d.czhi_h, d.czhi_l);
  split(q.diag, d.diag_h, d.diag_l);
  return d;
}

// the mixed form evaluates its outer residual in double-float arithmetic unless
// FERROX_DF_RESID=0 is set in the environment (FP64 residual; for comparisons)
bool df_resid_enabled() {
  const char* v = std::getenv("FERROX_DF_RESID");
  return !(v && v[0] == '0');
}

// residual instantiation for the stack's carriers: 0 none, 1 Boltzmann only, 2 with
// Fermi-Dirac planes
int carrier_kind(const ferrox_ctx* c) {
  if (!c->has_sc) return 0;
  for (const auto& p : c->planes)
    if (p.sc && p.fd) return 2;
  return 1;
}

struct NoWrap {
  template <typename F>
  void operator()(int, double, F&& f) const { f(); }
};

// Algorithmic bytes of one launch (each array element the method needs read or
// written once), for the profiler's per-class bandwidth figures.  T-sized
// multigrid arrays; FP64 state and right-hand side.
template <typename T>
double sweep_bytes(const ferrox_ctx* c, const LevelDesc& L) {
  // one colour: the other colour's e (read), own r (read), own e (write), own s (SC)
  return 0.5 * (double)L.ncell * sizeof(T) * (c->shift ? 4.0 : 3.0);
}
template <typename T>
double restrict_bytes(const LevelDesc& F, const LevelDesc& Cc) {
  return (double)F.ncell * 2.0 * sizeof(T) + (double)Cc.ncell * sizeof(T);
}
template <typename T>
double prolong_bytes(const LevelDesc& F, const LevelDesc& Cc) {
  return (double)Cc.ncell * sizeof(T) + (double)F.ncell * 2.0 * sizeof(T);
}

// One V-cycle on the correction equation; `wrap(kind, launch)` lets the profiler
// bracket each launch with events (identity when capturing graphs).
// V-cycles per outer iteration (numerics.inner; 0 means 1; < 0: adaptive, see adapt_max)
int inner_cycles(const ferrox_ctx* c) { return c->num.inner > 1 ? c->num.inner : 1; }
// adaptive inner cycles: at most -inner V-cycles per outer iteration, the count
// chosen on the device after every FP64 residual (0: fixed count)
int adapt_max(const ferrox_ctx* c) { return c->num.inner < 0 ? -c->num.inner : 0; }

// Levels whose smoothing runs as fused red-black sweeps (one launch per full
// sweep, alternating between the level's array and e_alt): the level must take
// the fused kernel's tile, and the sweep count must be even so that the last
// sweep lands in the level's own array.
template <typename T>
bool rb_sweeps(const ferrox_ctx* c, int l, int nu) {
  return c->e_alt && nu % 2 == 0 && smooth_rb_tile<T>(c->lv[l], c->shift) > 0;
}

// kernels of one smoothing of level l with nu sweeps
int smoothing_launches(const ferrox_ctx* c, int l, int nu) {
  const bool rb = c->num.precision == FERROX_MIXED ? rb_sweeps<float>(c, l, nu)
                                                   : rb_sweeps<double>(c, l, nu);
  return rb ? nu : 2 * nu;
}

// first: the fine level starts from a zero correction; last: phi += e rides on
// the last fine-level sweep
// levels l0 .. L of one V-cycle (l0 = 1: the coarse part of the direct form)
template <typename T, typename W = NoWrap>
void enqueue_levels(ferrox_ctx* c, cudaStream_t s, W wrap, int l0, bool first, bool last) {
  MGArgs<T> a = mg_args<T>(c);
  // level 0's sweeps multiply by 1 / (diag + s), written with s by the residual
  MGArgs<T> a0 = a;
  a0.sinv = static_cast<const T*>(c->sinv0);
  auto sw_args = [&](int l) -> const MGArgs<T>& { return l == 0 ? a0 : a; };
  const int nu1 = c->num.nu1, nu2 = c->num.nu2;
  const int constant = 0;
  const int lt = c->tail_first, L = (int)c->lv.size() - 1;
  T* alt = static_cast<T*>(c->e_alt);
  for (int l = l0; l < lt; ++l) {
    const int ks = l == 0 ? FERROX_K_SMOOTH0 : FERROX_K_SMOOTHC;
    const double sb = sweep_bytes<T>(c, c->lv[l]);
    if (rb_sweeps<T>(c, l, nu1)) {
      T* own = a.e + c->lv[l].off;
      for (int sw = 0; sw < nu1; ++sw) {
        const int zero = sw == 0 && (first || l > 0);
        T* src = sw % 2 ? alt : own;
        T* dst = sw % 2 ? own : alt;
        wrap(ks, 2.0 * sb, [&] { launch_smooth_rb<T>(sw_args(l), c->lv[l], src, dst, zero, nullptr, s); });
      }
    } else {
      for (int sw = 0; sw < nu1; ++sw) {
        const int zero = sw == 0 && (first || l > 0);
        wrap(ks, sb, [&] { launch_smooth<T>(sw_args(l), c->lv[l], 0, zero, nullptr, s); });
        wrap(ks, sb, [&] { launch_smooth<T>(sw_args(l), c->lv[l], 1, 0, nullptr, s); });
      }
    }
    wrap(FERROX_K_RESTRICT, restrict_bytes<T>(c->lv[l], c->lv[l + 1]),
         [&] { launch_restrict<T>(a, c->lv[l], c->lv[l + 1], nu1, s); });
  }
  if (c->dense_wide_d) {
    // the whole tail as one exact solve of its first level, spread over the SMs
    const LevelDesc& B = c->lv[lt];
    // the inverse (n^2 elements) and the level's r in, e out
    const double n = (double)B.ncell;
    wrap(FERROX_K_TAIL, (n * n + 2.0 * n) * sizeof(T), [&] {
      launch_dense_solve<T>(static_cast<const T*>(c->dense_wide_d), (int)B.ncell, a.r + B.off,
                            a.e + B.off, s);
    });
  } else {
    TailArgs ta{c->lvt_d, L - lt + 1, c->tail_elems, c->lv[lt].off, nu1, nu2, c->num.bottom_sweeps,
                constant, c->dense_d, c->dense_lev, 0};
    double tb = 0.0;   // every tail level's r in and e out once (shared memory in between)
    for (int l = lt; l <= L; ++l) tb += 2.0 * (double)c->lv[l].ncell * sizeof(T);
    wrap(FERROX_K_TAIL, tb, [&] { launch_tail<T>(a, ta, c->tail_smem, s); });
  }
  const UpdateArgs upd{c->phi, c->stats_d, update_clamp(c)};
  for (int l = lt - 1; l >= l0; --l) {
    const int ks = l == 0 ? FERROX_K_SMOOTH0 : FERROX_K_SMOOTHC;
    // the tiled form where FP64 arithmetic bounds the launch: the fine level
    const bool tiled = sizeof(T) == sizeof(double) && l == 0;
    wrap(FERROX_K_PROLONG, prolong_bytes<T>(c->lv[l], c->lv[l + 1]),
         [&] { launch_prolong<T>(a, c->lv[l], c->lv[l + 1], constant, s, tiled); });
    const double sb = sweep_bytes<T>(c, c->lv[l]);
    const bool rb = rb_sweeps<T>(c, l, nu2);
    T* own = a.e + c->lv[l].off;
    for (int sw = 0; sw < nu2; ++sw) {
      const bool fuse = last && l == 0 && sw == nu2 - 1;   // phi += e folded into the last sweep
      // the fused update also reads and writes phi (FP64) of the swept cells
      if (rb) {
        const double ub = fuse ? (double)c->lv[0].ncell * 16.0 : 0.0;
        T* src = sw % 2 ? alt : own;
        T* dst = sw % 2 ? own : alt;
        wrap(ks, 2.0 * sb + ub,
             [&] { launch_smooth_rb<T>(sw_args(l), c->lv[l], src, dst, 0, fuse ? &upd : nullptr, s); });
      } else {
        const double ub = fuse ? 0.5 * (double)c->lv[0].ncell * 16.0 : 0.0;
        wrap(ks, sb, [&] { launch_smooth<T>(sw_args(l), c->lv[l], 0, 0, nullptr, s); });
        wrap(ks, sb + ub, [&] { launch_smooth<T>(sw_args(l), c->lv[l], 1, 0, fuse ? &upd : nullptr, s); });
      }
    }
  }
}

template <typename T, typename W = NoWrap>
void enqueue_vcycle(ferrox_ctx* c, cudaStream_t s, W wrap = W(), bool first = true,
                    bool last = true) {
  enqueue_levels<T>(c, s, wrap, 0, first, last);
}

// ---- direct FP64 form: V-cycles on phi itself -------------------------------------
// The fine level relaxes A phi = b in place (b holds the whole right-hand side:
// the TDGL update writes its planes, launch_static_b the electrode lift of the
// others); the residual b - A phi after the pre-smoothing is restricted and its
// norm decides convergence in the same kernel, so no separate residual pass,
// correction array or update runs on the fine level.  Used for FP64 stacks
// without carriers (no Newton shift), one V-cycle per check and a fine level
// coarsened in all three directions (the tiled prolongation writes phi).
bool direct_form(const ferrox_ctx* c) {
  return c->num.precision == FERROX_FP64 && !c->has_sc && c->num.inner <= 1 &&
         c->num.inner >= 0 && c->tail_first >= 1 && c->lv.size() >= 2 && c->lv[0].crx &&
         c->lv[0].cry && c->lv[0].crz;
}

MGArgs<double> fine_args(ferrox_ctx* c) {
  MGArgs<double> a = mg_args<double>(c);
  a.e = c->phi;   // level 0 has arena offset 0
  a.r = c->b;
  a.s = nullptr;
  return a;
}

// nu1 red/black sweep pairs on phi; zst: honour the solve's b = 0 flag (phi = 0).
// The sweeps read b / diag (written once per solve by the prologue) with the
// level's coefficients divided by the diagonal.
template <typename W>
void enqueue_fine_sweeps(ferrox_ctx* c, cudaStream_t s, W wrap, int nu, const DevStats* zst) {
  MGArgs<double> fa = fine_args(c);
  fa.r = c->bs;
  fa.coef = c->coef0s;
  for (int sw = 0; sw < nu; ++sw) {
    const double sb = sweep_bytes<double>(c, c->lv[0]);
    wrap(FERROX_K_SMOOTH0, sb, [&] { launch_smooth_scaled(fa, c->lv[0], 0, s, zst); });
    wrap(FERROX_K_SMOOTH0, sb, [&] { launch_smooth_scaled(fa, c->lv[0], 1, s, zst); });
  }
}

// kernels of one loop iteration of the direct form (= one V-cycle)
int vcycle_launches(const ferrox_ctx* c);

template <typename W>
void enqueue_check(ferrox_ctx* c, cudaStream_t s, W wrap, int first, int set_cond,
                   unsigned long long handle) {
  CheckArgs ck{};
  ck.partials = c->partials_d;
  ck.stats = c->stats_d;
  ck.tol = c->num.tol;
  ck.max_cycles = c->num.max_cycles;
  ck.first = first;
  ck.set_cond = set_cond;
  ck.launches_per_cycle = vcycle_launches(c);
  ck.cond_handle = handle;
  ck.first_launches = 2 * c->num.nu1 + 2;   // b / diag, pre-smoothing, the check
  const MGArgs<double> fa = fine_args(c);
  double* rc = static_cast<double*>(c->r_arena);
  // phi and b of the fine level read, the coarse residual written
  const double rb = (double)c->lv[0].ncell * 16.0 + (double)c->lv[1].ncell * 8.0;
  wrap(FERROX_K_RESID, rb, [&] { launch_restrict_check(fa, rc, c->lv[0], c->lv[1], c->num.nu1, ck, s); });
}

// prologue of a solve: pre-smoothing and the first check
template <typename W = NoWrap>
void enqueue_direct_prologue(ferrox_ctx* c, cudaStream_t s, W wrap, int set_cond,
                             unsigned long long handle) {
  const double nb = (double)c->lv[0].ncell * 16.0;
  wrap(FERROX_K_COPY, nb, [&] { launch_scale_rhs(c->b, c->coef0, c->nx, c->ny, c->nz, c->bs, s); });
  enqueue_fine_sweeps(c, s, wrap, c->num.nu1, nullptr);
  enqueue_check(c, s, wrap, 1, set_cond, handle);
}

// one loop iteration: the coarse levels, their correction prolongated into phi,
// post-smoothing, the next pre-smoothing and check
template <typename W = NoWrap>
void enqueue_direct_cycle(ferrox_ctx* c, cudaStream_t s, W wrap, int set_cond,
                          unsigned long long handle) {
  enqueue_levels<double>(c, s, wrap, 1, true, false);
  MGArgs<double> a = mg_args<double>(c);
  wrap(FERROX_K_PROLONG, prolong_bytes<double>(c->lv[0], c->lv[1]),
       [&] { launch_prolong<double>(a, c->lv[0], c->lv[1], 0, s, true, c->phi); });
  enqueue_fine_sweeps(c, s, wrap, c->num.nu2, c->stats_d);
  enqueue_fine_sweeps(c, s, wrap, c->num.nu1, c->stats_d);
  enqueue_check(c, s, wrap, 0, set_cond, handle);
}

// the V-cycles of one outer iteration
template <typename T, typename W = NoWrap>
void enqueue_cycles(ferrox_ctx* c, cudaStream_t s, W wrap = W()) {
  const int q = inner_cycles(c);
  for (int i = 0; i < q; ++i) enqueue_vcycle<T>(c, s, wrap, i == 0, i == q - 1);
}

// the fine-level update is a separate kernel only when it cannot ride on a sweep
bool separate_update(const ferrox_ctx* c) {
  return c->tail_first == 0 || c->num.nu2 == 0 || adapt_max(c) > 0;
}

// kernels launched by one outer iteration: V-cycle, (update), residual
int vcycle_launches(const ferrox_ctx* c) {
  int n = 1;   // the tail or the dense bottom solve
  for (int l = 0; l < c->tail_first; ++l)
    n += smoothing_launches(c, l, c->num.nu1) + 1 + 1 + smoothing_launches(c, l, c->num.nu2);
  return n;
}

int launches_per_cycle(const ferrox_ctx* c) {
  if (c->direct) return vcycle_launches(c);
  if (adapt_max(c) > 0) return 1 + 1 + 1;   // arm, update, resid (V-cycles counted on the device)
  return inner_cycles(c) * vcycle_launches(c) + (separate_update(c) ? 1 : 0) + 1;
}

int tdgl_launches(const ferrox_ctx* c) { return c->ncomp == 3 ? 2 : 1; }

template <typename T>
void enqueue_resid(ferrox_ctx* c, cudaStream_t s, int first, int set_cond,
                   unsigned long long handle, const double* reject_ref = nullptr,
                   unsigned long long reject_handle = 0) {
  ResidArgs a{};
  a.reject_ref = reject_ref;
  a.reject_handle = reject_handle;
  a.phi = c->phi; a.b = c->b; a.planes = c->planes_d; a.coef0 = c->coef0; a.params = c->params_d;
  a.nx = c->nx; a.ny = c->ny; a.nz = c->nz;
  a.r_out = c->r_arena;
  a.s_out = c->shift ? c->s_arena : nullptr;
  a.sinv_out = c->shift ? c->sinv0 : nullptr;
  a.carriers = carrier_kind(c);
  a.coef_df = c->df_resid ? c->coef_df : nullptr;
  a.partials = c->partials_d;
  a.kchunk = c->df_resid ? c->resid_kchunk_df : c->resid_kchunk;
  a.stats = c->stats_d;
  a.tol = c->num.tol;
  a.max_cycles = c->num.max_cycles;
  a.first = first;
  a.set_cond = set_cond;
  a.cond_handle = handle;
  a.launches_per_cycle = launches_per_cycle(c);
  a.adapt_max = adapt_max(c);
  a.launches_per_vcycle = vcycle_launches(c) + 1;   // + the countdown
  a.inner_fixed = inner_cycles(c);
  launch_resid<T>(a, s);
}

template <typename T>
void enqueue_update(ferrox_ctx* c, cudaStream_t s) {
  if (!separate_update(c)) return;
  T* e = static_cast<T*>(c->e_arena);
  launch_update<T>(c->phi, e, (long long)c->nx * c->ny * c->nz, c->stats_d, update_clamp(c), s,
                   adapt_max(c) > 0 ? e : nullptr);
}

// The FP32 TDGL coefficients of each plane (see PlaneF32): the force's
// coefficients rounded to FP32, d2z rewritten on differences, and the right-hand
// side b = -(Pf(k + 1/2) - Pf(k - 1/2)) h/eps0 folded into weights of P_{k-1},
// P_k, P_{k+1} (the face value is P_k on an electrode face).
std::vector<PlaneF32> planes_f32(const std::vector<PlaneTDGL>& pl, double b_scale) {
  const int nz = (int)pl.size();
  std::vector<PlaneF32> out(nz);
  for (int k = 0; k < nz; ++k) {
    const PlaneTDGL& p = pl[k];
    PlaneF32& q = out[k];
    q.fe = p.fe;
    q.alpha = (float)p.alpha; q.beta = (float)p.beta; q.gamma = (float)p.gamma;
    q.g11 = (float)p.g11; q.g44 = (float)p.g44; q.Gamma = (float)p.Gamma;
    q.wz_dn = (float)p.wz_dn; q.wz_up = (float)p.wz_up; q.wz_sum = (float)(p.wz_dn + p.wz_c + p.wz_up);
    q.fw_L = (float)p.fw_L; q.fw_R = (float)p.fw_R; q.fpc = (float)p.fpc;
    q.c_dn = k == 0 ? 0.0 : b_scale * p.fw_R;
    q.c_0 = b_scale * ((k == 0 ? 1.0 : p.fw_L) - (k == nz - 1 ? 1.0 : pl[k + 1].fw_R));
    q.c_up = k == nz - 1 ? 0.0 : -b_scale * pl[k + 1].fw_L;
  }
  return out;
}

TDGLArgs tdgl_args(ferrox_ctx* c, int mode) {
  TDGLArgs a{};
  a.phi = c->phi; a.b = c->b; a.planes = c->planes_d; a.params = c->params_d;
  a.nx = c->nx; a.ny = c->ny; a.nz = c->nz; a.ncomp = c->ncomp;
  a.kd_lo = c->kd_lo; a.kd_hi = c->kd_hi;
  a.dt = c->num.dt; a.inv_h = 1.0 / c->h; a.inv_h2 = 1.0 / (c->h * c->h);
  a.b_scale = c->h / kEps0;
  a.mode = mode;
  a.F_store = c->Fbuf;
  if (mode == 0 || mode == 1 || mode == 3) { a.P_in = c->P; a.P_out = c->Pbuf; a.P_base = nullptr; }
  else { a.P_in = c->Pbuf; a.P_out = c->P; a.P_base = c->P; }
  a.planes_f32 = c->planes_f32_d;
  a.dtf = (float)a.dt; a.inv_hf = (float)a.inv_h; a.inv_h2f = (float)a.inv_h2;
  return a;
}

// copy the new polarization (FE planes of every component) back to the caller's array
cudaError_t enqueue_copy_back(ferrox_ctx* c, cudaStream_t s) {
  const long long plane = (long long)c->nx * c->ny, N = plane * c->nz;
  const size_t off = (size_t)c->fe_lo * plane;
  const size_t cnt = (size_t)(c->fe_hi - c->fe_lo + 1) * plane;
  for (int q = 0; q < c->ncomp; ++q) {
    cudaError_t e = cudaMemcpyAsync(c->P + q * N + off, c->Pbuf + q * N + off, cnt * sizeof(double),
                                    cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// resid (sets the condition) -> WHILE { V-cycle; update; resid } on the capturing stream s.
// guard: phi holds a learned correction of the guess saved in phi_guess; the first
// residual rejects it unless it lowered ||r||, and then IF { phi = guess; resid } runs.
template <typename T>
ferrox_status capture_solve(ferrox_ctx* ctx, cudaStream_t s, bool guard = false) {
  cudaStreamCaptureStatus st;
  cudaGraph_t g;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  FX_CK(cudaStreamGetCaptureInfo(s, &st, nullptr, &g, nullptr, nullptr, nullptr));
  cudaGraphConditionalHandle h;
  FX_CK(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
  if (guard) {
    cudaGraphConditionalHandle hr;
    FX_CK(cudaGraphConditionalHandleCreate(&hr, g, 0, cudaGraphCondAssignDefault));
    enqueue_resid<T>(ctx, s, 1, 1, (unsigned long long)h, ctx->nn_scale + 1,
                     (unsigned long long)hr);
    FX_CK(cudaGetLastError());
    FX_CK(cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, nullptr, &nd));
    cudaGraphNodeParams ip = {cudaGraphNodeTypeConditional};
    ip.conditional.handle = hr;
    ip.conditional.type = cudaGraphCondTypeIf;
    ip.conditional.size = 1;
    cudaGraphNode_t ifn;
    FX_CK(cudaGraphAddNode(&ifn, g, deps, nullptr, nd, &ip));
    FX_CK(cudaStreamBeginCaptureToGraph(ctx->cap2, ip.conditional.phGraph_out[0], nullptr, nullptr,
                                        0, cudaStreamCaptureModeRelaxed));
    FX_CK(cudaMemcpyAsync(ctx->phi, ctx->phi_guess,
                          (size_t)ctx->nx * ctx->ny * ctx->nz * sizeof(double),
                          cudaMemcpyDeviceToDevice, ctx->cap2));
    enqueue_resid<T>(ctx, ctx->cap2, 1, 1, (unsigned long long)h);
    FX_CK(cudaGetLastError());
    cudaGraph_t if_out;
    FX_CK(cudaStreamEndCapture(ctx->cap2, &if_out));
    FX_CK(cudaStreamUpdateCaptureDependencies(s, &ifn, nullptr, 1, cudaStreamSetCaptureDependencies));
  } else if (ctx->direct) {
    enqueue_direct_prologue(ctx, s, NoWrap(), 1, (unsigned long long)h);
  } else {
    enqueue_resid<T>(ctx, s, 1, 1, (unsigned long long)h);
  }
  FX_CK(cudaGetLastError());
  FX_CK(cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, nullptr, &nd));
  cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cn;
  FX_CK(cudaGraphAddNode(&cn, g, deps, nullptr, nd, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  FX_CK(cudaStreamBeginCaptureToGraph(ctx->cap2, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeRelaxed));
  if (ctx->direct) {
    enqueue_direct_cycle(ctx, ctx->cap2, NoWrap(), 1, (unsigned long long)h);
    FX_CK(cudaGetLastError());
    cudaGraph_t body_out;
    FX_CK(cudaStreamEndCapture(ctx->cap2, &body_out));
    FX_CK(cudaStreamUpdateCaptureDependencies(s, &cn, nullptr, 1, cudaStreamSetCaptureDependencies));
    return FERROX_OK;
  }
  if (adapt_max(ctx) > 0) {
    // arm -> WHILE { V-cycle continuing the correction; countdown } (count set by the resid)
    cudaGraphConditionalHandle hi;
    FX_CK(cudaGraphConditionalHandleCreate(&hi, body, 0, 0));
    launch_inner_arm(ctx->stats_d, (unsigned long long)hi, ctx->cap2);
    FX_CK(cudaGetLastError());
    const cudaGraphNode_t* bdeps = nullptr;
    size_t bnd = 0;
    cudaGraph_t bg;
    FX_CK(cudaStreamGetCaptureInfo(ctx->cap2, &st, nullptr, &bg, &bdeps, nullptr, &bnd));
    cudaGraphNodeParams ip = {cudaGraphNodeTypeConditional};
    ip.conditional.handle = hi;
    ip.conditional.type = cudaGraphCondTypeWhile;
    ip.conditional.size = 1;
    cudaGraphNode_t icn;
    FX_CK(cudaGraphAddNode(&icn, bg, bdeps, nullptr, bnd, &ip));
    FX_CK(cudaStreamBeginCaptureToGraph(ctx->cap3, ip.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                        cudaStreamCaptureModeRelaxed));
    enqueue_vcycle<T>(ctx, ctx->cap3, NoWrap(), false, false);
    launch_inner_countdown(ctx->stats_d, (unsigned long long)hi, ctx->cap3);
    FX_CK(cudaGetLastError());
    cudaGraph_t ibody_out;
    FX_CK(cudaStreamEndCapture(ctx->cap3, &ibody_out));
    FX_CK(cudaStreamUpdateCaptureDependencies(ctx->cap2, &icn, nullptr, 1, cudaStreamSetCaptureDependencies));
  } else {
    enqueue_cycles<T>(ctx, ctx->cap2);
  }
  enqueue_update<T>(ctx, ctx->cap2);
  enqueue_resid<T>(ctx, ctx->cap2, 0, 1, (unsigned long long)h);
  FX_CK(cudaGetLastError());
  cudaGraph_t body_out;
  FX_CK(cudaStreamEndCapture(ctx->cap2, &body_out));
  FX_CK(cudaStreamUpdateCaptureDependencies(s, &cn, nullptr, 1, cudaStreamSetCaptureDependencies));
  return FERROX_OK;
}

template <typename T>
ferrox_status build_graphs_t(ferrox_ctx* ctx) {
  cudaStream_t s = ctx->cap1;
  ferrox_status rc;
  // solve only
  FX_CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
  if ((rc = capture_solve<T>(ctx, s)) != FERROX_OK) return rc;
  FX_CK(cudaStreamEndCapture(s, &ctx->gr_solve));
  FX_CK(cudaGraphInstantiate(&ctx->ge_solve, ctx->gr_solve, 0));
  // TDGL update only (Step 1a)
  FX_CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
  launch_tdgl(tdgl_args(ctx, 0), s);
  FX_CK(enqueue_copy_back(ctx, s));
  FX_CK(cudaStreamEndCapture(s, &ctx->gr_tdgl));
  FX_CK(cudaGraphInstantiate(&ctx->ge_tdgl, ctx->gr_tdgl, 0));
  // full time step
  FX_CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
  const long long N = (long long)ctx->nx * ctx->ny * ctx->nz;
  if (ctx->num.order == 1) {
    launch_tdgl(tdgl_args(ctx, 0), s);                 // Step 1a
    FX_CK(enqueue_copy_back(ctx, s));
    if (ctx->num.guess == 1) launch_extrapolate(ctx->phi, ctx->phi_prev, N, s);
    if ((rc = capture_solve<T>(ctx, s)) != FERROX_OK) return rc;   // Step 1b
  } else {
    launch_tdgl(tdgl_args(ctx, 1), s);                 // Step 1a (P* to scratch, f(P^n) kept)
    if (ctx->num.guess == 1) launch_extrapolate(ctx->phi, ctx->phi_prev, N, s);
    if ((rc = capture_solve<T>(ctx, s)) != FERROX_OK) return rc;   // Step 1b: Phi*
    launch_tdgl(tdgl_args(ctx, 2), s);                 // Step 2a: P^{n+1} into the caller's P
    if ((rc = capture_solve<T>(ctx, s)) != FERROX_OK) return rc;   // Step 2b
  }
  launch_stats_step(ctx->stats_d, 1,
                    tdgl_launches(ctx) * ctx->num.order + 1 + (ctx->num.guess == 1 ? 1 : 0), s);
  FX_CK(cudaGetLastError());
  FX_CK(cudaStreamEndCapture(s, &ctx->gr_step));
  FX_CK(cudaGraphInstantiate(&ctx->ge_step, ctx->gr_step, 0));
  return FERROX_OK;
}

// ---- learned warm start --------------------------------------------------------------------

// restricted initial residual -> network features (into x) and its rms (nn_scale)
template <typename T>
void enqueue_nn_features(ferrox_ctx* c, cudaStream_t s, __nv_bfloat16* x) {
  ResidArgs a{};
  a.phi = c->phi; a.b = c->b; a.planes = c->planes_d; a.coef0 = c->coef0; a.params = c->params_d;
  a.nx = c->nx; a.ny = c->ny; a.nz = c->nz;
  a.r_out = c->r_arena;
  a.s_out = c->shift ? c->s_arena : nullptr;
  a.sinv_out = c->shift ? c->sinv0 : nullptr;
  a.carriers = carrier_kind(c);
  a.coef_df = c->df_resid ? c->coef_df : nullptr;
  a.stats = c->stats_d;
  a.partials = c->partials_d;
  a.norm_out = c->nn_scale + 1;   // ||r|| of the guess, for the check of the correction
  a.kchunk = c->df_resid ? c->resid_kchunk_df : c->resid_kchunk;
  launch_resid<T>(a, s);
  T* r = static_cast<T*>(c->r_arena);
  nn_bridge_restrict<T>(r, c->lv, c->nn_level, s);
  nn_bridge_scale<T>(r, c->lv[c->nn_level], c->nn_scale, s);
  nn_bridge_features<T>(r, c->lv[c->nn_level], c->nn_pf, c->nn_scale, c->params_d, x, s);
}

// network prediction of the coarse error, prolongated and added to phi
template <typename T>
void enqueue_nn_prelude(ferrox_ctx* c, cudaStream_t s) {
  cudaMemcpyAsync(c->phi_guess, c->phi, (size_t)c->nx * c->ny * c->nz * sizeof(double),
                  cudaMemcpyDeviceToDevice, s);
  enqueue_nn_features<T>(c, s, nn_input(c->nn));
  nn_run_forward(c->nn, s);
  const size_t tsz = sizeof(T);
  const int lv = c->nn_level;
  cudaMemsetAsync(c->e_arena, 0, (size_t)c->lv[lv].off * tsz, s);
  T* e = static_cast<T*>(c->e_arena);
  nn_bridge_apply<T>(nn_output(c->nn), c->lv[lv], c->nn_scale, e, s);
  MGArgs<T> a = mg_args<T>(c);
  for (int l = lv - 1; l >= 0; --l) launch_prolong<T>(a, c->lv[l], c->lv[l + 1], 0, s);
  launch_update<T>(c->phi, e, (long long)c->nx * c->ny * c->nz, c->nn_stats, update_clamp(c), s,
                   adapt_max(c) > 0 ? e : nullptr);
}

template <typename T>
ferrox_status capture_nn_step(ferrox_ctx* ctx, cudaStream_t s) {
  ferrox_status rc;
  const long long N = (long long)ctx->nx * ctx->ny * ctx->nz;
  if (ctx->num.order == 1) {
    launch_tdgl(tdgl_args(ctx, 0), s);
    FX_CK(enqueue_copy_back(ctx, s));
    if (ctx->num.guess == 1) launch_extrapolate(ctx->phi, ctx->phi_prev, N, s);
    enqueue_nn_prelude<T>(ctx, s);
    if ((rc = capture_solve<T>(ctx, s, true)) != FERROX_OK) return rc;
  } else {
    launch_tdgl(tdgl_args(ctx, 1), s);
    if (ctx->num.guess == 1) launch_extrapolate(ctx->phi, ctx->phi_prev, N, s);
    enqueue_nn_prelude<T>(ctx, s);
    if ((rc = capture_solve<T>(ctx, s, true)) != FERROX_OK) return rc;
    launch_tdgl(tdgl_args(ctx, 2), s);
    if ((rc = capture_solve<T>(ctx, s)) != FERROX_OK) return rc;
  }
  launch_stats_step(ctx->stats_d, 1, 0, s);
  FX_CK(cudaGetLastError());
  return FERROX_OK;
}

// The learned step runs the defect-correction form (its first residual is the
// check of the correction), also where plain FP64 solves use the direct form.
template <typename T>
ferrox_status build_nn_graph_t(ferrox_ctx* ctx) {
  cudaStream_t s = ctx->cap1;
  FX_CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
  const bool direct = ctx->direct;
  ctx->direct = false;
  const ferrox_status rc = capture_nn_step<T>(ctx, s);
  ctx->direct = direct;
  if (rc != FERROX_OK) return rc;
  FX_CK(cudaStreamEndCapture(s, &ctx->gr_step_nn));
  FX_CK(cudaGraphInstantiate(&ctx->ge_step_nn, ctx->gr_step_nn, 0));
  return FERROX_OK;
}

// one step that also records a (features, target) snapshot into the network's store
template <typename T>
ferrox_status collect_step_t(ferrox_ctx* ctx) {
  cudaStream_t s = ctx->stream;
  const long long N = (long long)ctx->nx * ctx->ny * ctx->nz;
  if (ctx->num.order != 1) return fail(ctx, FERROX_EINVAL, "snapshot collection runs order-1 steps");
  const int slot = nn_next_slot(ctx->nn);
  const LevelDesc& L = ctx->lv[ctx->nn_level];
  launch_tdgl(tdgl_args(ctx, 0), s);
  FX_CK(enqueue_copy_back(ctx, s));
  if (ctx->num.guess == 1) launch_extrapolate(ctx->phi, ctx->phi_prev, N, s);
  enqueue_nn_features<T>(ctx, s, nn_snap_x(ctx->nn) + (size_t)slot * L.ncell * 16);
  FX_CK(cudaMemcpyAsync(ctx->phi_guess, ctx->phi, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  FX_CK(cudaGraphLaunch(ctx->ge_solve, s));
  T* e = static_cast<T*>(ctx->e_arena);
  nn_bridge_guess_error<T>(ctx->phi, ctx->phi_guess, N, e, s);
  nn_bridge_restrict<T>(e, ctx->lv, ctx->nn_level, s);
  nn_bridge_target<T>(e, L, ctx->nn_scale, nn_snap_t(ctx->nn) + (size_t)slot * L.ncell, s);
  launch_stats_step(ctx->stats_d, 1, 0, s);
  FX_CK(cudaGetLastError());
  nn_note_snapshots(ctx->nn, 1);
  return FERROX_OK;
}

// ---- eager, event-timed step (per-kernel breakdown) -------------------------------------
struct EventTimer {
  cudaStream_t s;
  struct Rec {
    int kind;
    double bytes;
    cudaEvent_t a, b;
  };
  std::vector<Rec> rec;
  template <typename F>
  void operator()(int kind, double bytes, F&& f) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, s);
    f();
    cudaEventRecord(b, s);
    rec.push_back({kind, bytes, a, b});
  }
};

// algorithmic bytes of the step-level launches (FP64 state; T-sized residual)
struct StepBytes {
  double resid, tdgl, copy_back, extrap, update;
};

template <typename T>
StepBytes step_bytes(const ferrox_ctx* c) {
  const double plane = (double)c->nx * c->ny, N = plane * c->nz;
  double dyn = 0.0, fe = 0.0, sc = 0.0;
  for (const auto& p : c->planes) {
    dyn += p.b_dyn ? plane : 0.0;
    fe += p.fe ? plane : 0.0;
  }
  for (const auto& L : c->layers) sc += L.kind == FERROX_SC ? plane * L.ncells : 0.0;
  StepBytes b;
  // phi read, b read on the planes the TDGL update writes, r written, s written (SC)
  b.resid = N * (8.0 + sizeof(T)) + dyn * 8.0 + sc * sizeof(T);
  // P (all components) and phi read, new P written; b written on the dynamic planes
  b.tdgl = fe * c->ncomp * 16.0 + fe * 8.0 + dyn * 8.0;
  b.copy_back = fe * c->ncomp * 16.0;
  b.extrap = N * 24.0;
  b.update = N * (sizeof(T) + 16.0);
  return b;
}

// Launches between two host synchronisations queue up behind a short delay
// kernel (about 2 ms of SM clock, untimed), so the device runs them back to back
// and each event pair times its kernel rather than the host's launch rate.
constexpr long long kProfileGateCycles = 4000000;

template <typename T>
ferrox_status profile_step_t(ferrox_ctx* ctx, double* ms, int* count, double* bytes) {
  cudaStream_t s = ctx->stream;
  EventTimer tm{s, {}};
  const StepBytes sb = step_bytes<T>(ctx);
  auto gate = [&]() { launch_delay(kProfileGateCycles, s); };
  auto solve = [&]() -> ferrox_status {
    gate();
    if (ctx->direct) {
      enqueue_direct_prologue(ctx, s, std::ref(tm), 0, 0ULL);
      for (int guard = 0; guard <= ctx->num.max_cycles + 1; ++guard) {
        FX_CK(cudaMemcpyAsync(ctx->host_pinned, reinterpret_cast<char*>(ctx->stats_d) +
                                                    offsetof(DevStats, last_cond),
                              sizeof(int), cudaMemcpyDeviceToHost, s));
        FX_CK(cudaStreamSynchronize(s));
        int cond;
        std::memcpy(&cond, ctx->host_pinned, sizeof(int));
        if (!cond) break;
        gate();
        enqueue_direct_cycle(ctx, s, std::ref(tm), 0, 0ULL);
      }
      return FERROX_OK;
    }
    tm(FERROX_K_RESID, sb.resid, [&] { enqueue_resid<T>(ctx, s, 1, 0, 0ULL); });
    for (int guard = 0; guard <= ctx->num.max_cycles + 1; ++guard) {
      FX_CK(cudaMemcpyAsync(ctx->host_pinned, reinterpret_cast<char*>(ctx->stats_d) +
                                                  offsetof(DevStats, last_cond),
                            sizeof(int), cudaMemcpyDeviceToHost, s));
      FX_CK(cudaStreamSynchronize(s));
      int cond;
      std::memcpy(&cond, ctx->host_pinned, sizeof(int));
      if (!cond) break;
      if (adapt_max(ctx) > 0) {
        FX_CK(cudaMemcpyAsync(ctx->host_pinned, reinterpret_cast<char*>(ctx->stats_d) +
                                                    offsetof(DevStats, inner_k),
                              sizeof(int), cudaMemcpyDeviceToHost, s));
        FX_CK(cudaStreamSynchronize(s));
        int k;
        std::memcpy(&k, ctx->host_pinned, sizeof(int));
        gate();
        for (int i = 0; i < k; ++i) enqueue_vcycle<T>(ctx, s, std::ref(tm), false, false);
      } else {
        gate();
        enqueue_cycles<T>(ctx, s, std::ref(tm));
      }
      if (separate_update(ctx)) tm(FERROX_K_UPDATE, sb.update, [&] { enqueue_update<T>(ctx, s); });
      tm(FERROX_K_RESID, sb.resid, [&] { enqueue_resid<T>(ctx, s, 0, 0, 0ULL); });
    }
    return FERROX_OK;
  };
  ferrox_status rc;
  const long long N = (long long)ctx->nx * ctx->ny * ctx->nz;
  if (ctx->num.order == 1) {
    gate();
    tm(FERROX_K_TDGL, sb.tdgl, [&] { launch_tdgl(tdgl_args(ctx, 0), s); });
    tm(FERROX_K_COPY, sb.copy_back, [&] { enqueue_copy_back(ctx, s); });
    if (ctx->num.guess == 1)
      tm(FERROX_K_COPY, sb.extrap, [&] { launch_extrapolate(ctx->phi, ctx->phi_prev, N, s); });
    if ((rc = solve()) != FERROX_OK) return rc;
  } else {
    // order 2: the predictor also stores f (8 B per FE cell and component); the
    // corrector reads it and the base P
    gate();
    tm(FERROX_K_TDGL, sb.tdgl + sb.copy_back * 0.5, [&] { launch_tdgl(tdgl_args(ctx, 1), s); });
    if (ctx->num.guess == 1)
      tm(FERROX_K_COPY, sb.extrap, [&] { launch_extrapolate(ctx->phi, ctx->phi_prev, N, s); });
    if ((rc = solve()) != FERROX_OK) return rc;
    gate();
    tm(FERROX_K_TDGL, sb.tdgl + sb.copy_back, [&] { launch_tdgl(tdgl_args(ctx, 2), s); });
    if ((rc = solve()) != FERROX_OK) return rc;
  }
  launch_stats_step(ctx->stats_d, 1,
                    tdgl_launches(ctx) * ctx->num.order + 1 + (ctx->num.guess == 1 ? 1 : 0), s);
  FX_CK(cudaGetLastError());
  FX_CK(cudaStreamSynchronize(s));
  for (int k = 0; k < FERROX_K_COUNT; ++k) {
    ms[k] = 0.0;
    count[k] = 0;
    if (bytes) bytes[k] = 0.0;
  }
  for (auto& r : tm.rec) {
    float t = 0.f;
    cudaEventElapsedTime(&t, r.a, r.b);
    ms[r.kind] += t;
    count[r.kind] += 1;
    if (bytes) bytes[r.kind] += r.bytes;
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  return FERROX_OK;
}

void release(ferrox_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  cudaGraphExec_t ge[4] = {c->ge_step, c->ge_solve, c->ge_tdgl, c->ge_step_nn};
  cudaGraph_t gr[4] = {c->gr_step, c->gr_solve, c->gr_tdgl, c->gr_step_nn};
  for (auto g : ge) if (g) cudaGraphExecDestroy(g);
  for (auto g : gr) if (g) cudaGraphDestroy(g);
  void* ptrs[] = {c->b, c->Pbuf, c->Fbuf, c->phi_prev, c->e_arena, c->e_alt, c->r_arena, c->s_arena, c->coef, c->coef0, c->coef0s, c->bs, c->sinv0, c->coef_df,
                  c->planes_d, c->planes_f32_d, c->lv_d, c->lvt_d, c->nn_scale, c->phi_guess, c->nn_pf, c->nn_stats, c->params_d, c->stats_d, c->partials_d, c->charge_d,
                  c->charge_part_d, c->dense_d, c->dense_wide_d};
  for (void* p : ptrs) if (p) cudaFree(p);
  if (c->host_pinned) cudaFreeHost(c->host_pinned);
  if (c->cap1) cudaStreamDestroy(c->cap1);
  if (c->cap2) cudaStreamDestroy(c->cap2);
  if (c->cap3) cudaStreamDestroy(c->cap3);
  delete c;
}

ferrox_status validate(const ferrox_geometry* g, const ferrox_numerics* n, const double* P,
                       const double* phi) {
  auto bad = [](const char* m) { return fail(nullptr, FERROX_EINVAL, m); };
  if (!g || !n || !P || !phi) return bad("null argument");
  if ((reinterpret_cast<uintptr_t>(P) | reinterpret_cast<uintptr_t>(phi)) % 8)
    return bad("state arrays must be 8-byte aligned");
  if (g->nx < 1 || g->ny < 1) return bad("nx, ny must be >= 1");
  if ((g->nx != 1 && g->nx % 2) || (g->ny != 1 && g->ny % 2))
    return bad("lateral sizes must be even or 1 (periodic red-black colouring)");
  if (!(g->h > 0.0)) return bad("h must be > 0");
  if (g->nlayers < 1 || !g->layers) return bad("no layers");
  if (g->ncomp != 1 && g->ncomp != 3) return bad("ncomp must be 1 or 3");
  if (g->pbc < 0 || g->pbc > 2) return bad("unknown P boundary condition");
  if (g->pbc == FERROX_PBC_LAMBDA && !(g->lambda >= 0.0)) return bad("lambda must be >= 0");
  int nz = 0, nfe = 0;
  for (int q = 0; q < g->nlayers; ++q) {
    const ferrox_layer& L = g->layers[q];
    if (L.ncells < 1) return bad("layer with ncells < 1");
    if (!(L.eps_r > 0.0)) return bad("eps_r must be > 0");
    if (L.kind < 0 || L.kind > 2) return bad("unknown layer kind");
    if (L.kind == FERROX_FE) nfe++;
    if (L.kind == FERROX_SC && !(L.T > 0.0)) return bad("semiconductor temperature must be > 0");
    if (L.kind == FERROX_SC && (L.N_A < 0 || L.N_D < 0 || L.n_i < 0)) return bad("negative density");
    if (L.kind == FERROX_SC && L.stats != FERROX_BOLTZMANN && L.stats != FERROX_FERMI_DIRAC)
      return bad("unknown carrier statistics");
    if (L.kind == FERROX_SC && L.stats == FERROX_FERMI_DIRAC &&
        !(L.m_e > 0.0 && L.m_p > 0.0 && L.E_g > 0.0))
      return bad("Fermi-Dirac carriers need m_e, m_p, E_g > 0");
    nz += L.ncells;
  }
  if (nz < 2) return bad("Nz must be >= 2");
  if (nfe == 0) return bad("the stack needs a ferroelectric layer");
  if (!(n->dt > 0.0)) return bad("dt must be > 0");
  if (n->order != 1 && n->order != 2) return bad("order must be 1 or 2");
  if (!(n->tol > 0.0)) return bad("tol must be > 0");
  if (n->nu1 < 1 || n->nu2 < 0) return bad("need nu1 >= 1 and nu2 >= 0");
  if (n->max_cycles < 1) return bad("max_cycles must be >= 1");
  if (n->nonlinear != FERROX_NEWTON && n->nonlinear != FERROX_FIXED_POINT)
    return bad("nonlinear must be FERROX_NEWTON or FERROX_FIXED_POINT");
  if (n->precision != FERROX_FP64 && n->precision != FERROX_MIXED &&
      n->precision != FERROX_FP64_DEFECT)
    return bad("unknown precision");
  if (n->bottom_sweeps < 0) return bad("bottom_sweeps must be >= 0");
  if (n->inner < -16 || n->inner > 16) return bad("inner must be in -16..16");
  if (n->guess != 0 && n->guess != 1) return bad("guess must be 0 or 1");
  if (n->tdgl_arith != FERROX_TDGL_FP64 && n->tdgl_arith != FERROX_TDGL_FP32)
    return bad("tdgl_arith must be FERROX_TDGL_FP64 or FERROX_TDGL_FP32");
  if (n->tdgl_arith == FERROX_TDGL_FP32 && (n->precision != FERROX_MIXED || g->ncomp != 1))
    return bad("FP32 TDGL arithmetic needs the mixed precision and one polarization component");
  return FERROX_OK;
}

}  // namespace

extern "C" {

ferrox_status ferrox_init_geometry(ferrox_ctx** out, const ferrox_geometry* geom,
                                   const ferrox_numerics* num, double* P_dev, double* phi_dev,
                                   void* cuda_stream) {
  if (!out) return fail(nullptr, FERROX_EINVAL, "null output pointer");
  *out = nullptr;
  ferrox_status rc = validate(geom, num, P_dev, phi_dev);
  if (rc != FERROX_OK) return rc;
  ferrox_ctx* ctx = new ferrox_ctx();
  ctx->nx = geom->nx; ctx->ny = geom->ny; ctx->h = geom->h; ctx->pbc = geom->pbc;
  ctx->lambda = geom->lambda; ctx->ncomp = geom->ncomp;
  ctx->layers.assign(geom->layers, geom->layers + geom->nlayers);
  ctx->nz = 0;
  for (auto& L : ctx->layers) ctx->nz += L.ncells;
  ctx->num = *num;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  ctx->P = P_dev;
  ctx->phi = phi_dev;
  if ((rc = build_planes(ctx)) != FERROX_OK) { ctx->err = g_init_error; release(ctx); return rc; }
  ctx->shift = ctx->has_sc && ctx->num.nonlinear == FERROX_NEWTON;
  build_levels(ctx);
  if (ctx->arena >= (1LL << 31)) {   // the multigrid kernels index the arenas with 32-bit integers
    release(ctx);
    return fail(nullptr, FERROX_EINVAL, "grid too large: the multigrid arenas exceed 2^31 elements");
  }

  const bool mixed = ctx->num.precision == FERROX_MIXED;
  const size_t tsz = mixed ? sizeof(float) : sizeof(double);
  plan_tail(ctx, tsz, true);
  {
    // residual grid: split the columns into z chunks (halving, at least 4 planes
    // each) until there are about four waves of blocks on 152 SMs
    const int bxy = ((ctx->nx + kResidBX - 1) / kResidBX) * ((ctx->ny + kResidBY - 1) / kResidBY);
    int zc = 1;
    while ((long long)bxy * zc < 4LL * 152 * 3 && ctx->nz / (2 * zc) >= 4) zc *= 2;
    ctx->resid_kchunk = (ctx->nz + zc - 1) / zc;
    ctx->resid_blocks = bxy * ((ctx->nz + ctx->resid_kchunk - 1) / ctx->resid_kchunk);
    // the double-float form: at least 8 planes per thread (its block reduction and
    // per-column set-up cost more than the FP64 form's), about two waves
    int zd = 1;
    while ((long long)bxy * zd < 2LL * 152 * 4 && ctx->nz / (2 * zd) >= 8) zd *= 2;
    ctx->resid_kchunk_df = (ctx->nz + zd - 1) / zd;
  }
  ctx->direct = direct_form(ctx);
  if (ctx->direct) {
    const dim3 g = check_grid(ctx->lv[1]);
    ctx->check_blocks = (int)(g.x * g.y * g.z);
  }
  const long long N = (long long)ctx->nx * ctx->ny * ctx->nz;
  auto cleanup = [&](ferrox_status s) { g_init_error = ctx->err; release(ctx); return s; };
#define FX_INIT_CK(call)                                                                     \
  do {                                                                                       \
    cudaError_t _e = (call);                                                                 \
    if (_e != cudaSuccess) {                                                                 \
      ctx->err = std::string(#call) + ": " + cudaGetErrorString(_e);                        \
      return cleanup(_e == cudaErrorMemoryAllocation ? FERROX_ENOMEM : FERROX_ECUDA);        \
    }                                                                                        \
  } while (0)
  FX_INIT_CK(cudaStreamCreateWithFlags(&ctx->cap1, cudaStreamNonBlocking));
  FX_INIT_CK(cudaStreamCreateWithFlags(&ctx->cap2, cudaStreamNonBlocking));
  FX_INIT_CK(cudaStreamCreateWithFlags(&ctx->cap3, cudaStreamNonBlocking));
  FX_INIT_CK(cudaMalloc(&ctx->b, N * sizeof(double)));
  FX_INIT_CK(cudaMalloc(&ctx->Pbuf, ctx->ncomp * N * sizeof(double)));
  if (ctx->num.order == 2) FX_INIT_CK(cudaMalloc(&ctx->Fbuf, ctx->ncomp * N * sizeof(double)));
  if (ctx->num.guess == 1) {
    FX_INIT_CK(cudaMalloc(&ctx->phi_prev, N * sizeof(double)));
    FX_INIT_CK(cudaMemset(ctx->phi_prev, 0, N * sizeof(double)));
  }
  FX_INIT_CK(cudaMalloc(&ctx->e_arena, ctx->arena * tsz));
  // FERROX_RB_SWEEPS=0 in the environment keeps the colour-by-colour sweeps
  // (same results; for comparing the two paths)
  const char* rb_env = std::getenv("FERROX_RB_SWEEPS");
  if (mixed && !(rb_env && rb_env[0] == '0')) {
    // the fused red-black sweeps alternate between a level's array and e_alt
    long long alt = 0;
    for (int l = 0; l < ctx->tail_first; ++l)
      if (smooth_rb_tile<float>(ctx->lv[l], ctx->shift) > 0) alt = std::max(alt, ctx->lv[l].ncell);
    if (alt > 0) {
      FX_INIT_CK(cudaMalloc(&ctx->e_alt, alt * tsz));
      FX_INIT_CK(smooth_rb_prepare<float>());
    }
  }
  FX_INIT_CK(cudaMalloc(&ctx->r_arena, ctx->arena * tsz));
  if (ctx->shift) FX_INIT_CK(cudaMalloc(&ctx->s_arena, ctx->arena * tsz));
  if (ctx->shift) FX_INIT_CK(cudaMalloc(&ctx->sinv0, ctx->lv[0].ncell * tsz));
  FX_INIT_CK(cudaMalloc(&ctx->planes_d, ctx->nz * sizeof(PlaneTDGL)));
  FX_INIT_CK(cudaMalloc(&ctx->lv_d, ctx->lv.size() * sizeof(LevelDesc)));
  FX_INIT_CK(cudaMalloc(&ctx->params_d, sizeof(DevParams)));
  FX_INIT_CK(cudaMalloc(&ctx->stats_d, sizeof(DevStats)));
  FX_INIT_CK(cudaMalloc(&ctx->partials_d, std::max(3 * (size_t)ctx->resid_blocks,
                                                    2 * (size_t)ctx->check_blocks) *
                                               sizeof(double)));
  FX_INIT_CK(cudaMalloc(&ctx->lvt_d, ctx->lv_tail.size() * sizeof(LevelDesc)));
  FX_INIT_CK(cudaMemcpy(ctx->lvt_d, ctx->lv_tail.data(), ctx->lv_tail.size() * sizeof(LevelDesc),
                        cudaMemcpyHostToDevice));
  FX_INIT_CK(mixed ? tail_prepare<float>(ctx->tail_smem) : tail_prepare<double>(ctx->tail_smem));
  FX_INIT_CK(cudaMalloc(&ctx->charge_d, 8 * sizeof(double)));
  FX_INIT_CK(cudaMalloc(&ctx->charge_part_d, 4 * 64 * sizeof(double)));
  FX_INIT_CK(cudaMallocHost(&ctx->host_pinned, 64 * sizeof(double)));
  auto c64 = level_coefficients<double>(ctx);
  FX_INIT_CK(cudaMalloc(&ctx->coef0, ctx->nz * sizeof(PlaneCoef<double>)));
  FX_INIT_CK(cudaMemcpy(ctx->coef0, c64.data(), ctx->nz * sizeof(PlaneCoef<double>),
                        cudaMemcpyHostToDevice));
  if (ctx->direct) {
    // the direct form's fine sweeps: couplings divided by the diagonal, b / diag
    std::vector<PlaneCoef<double>> cs(c64.begin(), c64.begin() + ctx->nz);
    for (auto& q : cs) {
      q.cx *= q.invdiag; q.cy *= q.invdiag; q.czlo *= q.invdiag; q.czhi *= q.invdiag;
      q.diag = 1.0; q.invdiag = 1.0;
    }
    FX_INIT_CK(cudaMalloc(&ctx->coef0s, ctx->nz * sizeof(PlaneCoef<double>)));
    FX_INIT_CK(cudaMemcpy(ctx->coef0s, cs.data(), ctx->nz * sizeof(PlaneCoef<double>), cudaMemcpyHostToDevice));
    FX_INIT_CK(cudaMalloc(&ctx->bs, N * sizeof(double)));
  }
  {
    // the same coefficients as double-float pairs: h = the nearest float, l = the
    // nearest float to the remainder
    std::vector<PlaneCoefDF> cdf(ctx->nz);
    for (int k = 0; k < ctx->nz; ++k) cdf[k] = split_coef_df(c64[k]);
    FX_INIT_CK(cudaMalloc(&ctx->coef_df, ctx->nz * sizeof(PlaneCoefDF)));
    FX_INIT_CK(cudaMemcpy(ctx->coef_df, cdf.data(), ctx->nz * sizeof(PlaneCoefDF),
                          cudaMemcpyHostToDevice));
    ctx->df_resid = mixed && df_resid_enabled();
  }
  ctx->dense_lev = dense_level(ctx);
  if (mixed) {
    auto c32 = level_coefficients<float>(ctx);
    FX_INIT_CK(cudaMalloc(&ctx->coef, c32.size() * sizeof(PlaneCoef<float>)));
    FX_INIT_CK(cudaMemcpy(ctx->coef, c32.data(), c32.size() * sizeof(PlaneCoef<float>),
                          cudaMemcpyHostToDevice));
    if (ctx->dense_lev >= 0) {
      const auto inv = dense_inverse<float>(c32, ctx->lv_tail[ctx->dense_lev]);
      FX_INIT_CK(cudaMalloc(&ctx->dense_d, inv.size() * sizeof(float)));
      FX_INIT_CK(cudaMemcpy(ctx->dense_d, inv.data(), inv.size() * sizeof(float),
                            cudaMemcpyHostToDevice));
    }
    const LevelDesc& T0 = ctx->lv_tail[0];
    if (!ctx->shift && T0.ncell > kDenseMax && T0.ncell <= kDenseWide) {
      const auto inv = dense_inverse<float>(c32, T0);
      FX_INIT_CK(cudaMalloc(&ctx->dense_wide_d, inv.size() * sizeof(float)));
      FX_INIT_CK(cudaMemcpy(ctx->dense_wide_d, inv.data(), inv.size() * sizeof(float),
                            cudaMemcpyHostToDevice));
    }
  } else {
    FX_INIT_CK(cudaMalloc(&ctx->coef, c64.size() * sizeof(PlaneCoef<double>)));
    FX_INIT_CK(cudaMemcpy(ctx->coef, c64.data(), c64.size() * sizeof(PlaneCoef<double>),
                          cudaMemcpyHostToDevice));
    const LevelDesc& T0 = ctx->lv_tail[0];
    if (!ctx->shift && T0.ncell > kDenseMax && T0.ncell <= kDenseWide) {
      const auto inv = dense_inverse<double>(c64, T0);
      FX_INIT_CK(cudaMalloc(&ctx->dense_wide_d, inv.size() * sizeof(double)));
      FX_INIT_CK(cudaMemcpy(ctx->dense_wide_d, inv.data(), inv.size() * sizeof(double),
                            cudaMemcpyHostToDevice));
    }
    if (ctx->dense_lev >= 0) {
      const auto inv = dense_inverse<double>(c64, ctx->lv_tail[ctx->dense_lev]);
      FX_INIT_CK(cudaMalloc(&ctx->dense_d, inv.size() * sizeof(double)));
      FX_INIT_CK(cudaMemcpy(ctx->dense_d, inv.data(), inv.size() * sizeof(double),
                            cudaMemcpyHostToDevice));
    }
  }
  FX_INIT_CK(cudaMemcpy(ctx->planes_d, ctx->planes.data(), ctx->nz * sizeof(PlaneTDGL),
                        cudaMemcpyHostToDevice));
  if (ctx->num.tdgl_arith == FERROX_TDGL_FP32) {
    const std::vector<PlaneF32> pf = planes_f32(ctx->planes, ctx->h / kEps0);
    FX_INIT_CK(cudaMalloc(&ctx->planes_f32_d, pf.size() * sizeof(PlaneF32)));
    FX_INIT_CK(cudaMemcpy(ctx->planes_f32_d, pf.data(), pf.size() * sizeof(PlaneF32), cudaMemcpyHostToDevice));
  }
  FX_INIT_CK(cudaMemcpy(ctx->lv_d, ctx->lv.data(), ctx->lv.size() * sizeof(LevelDesc),
                        cudaMemcpyHostToDevice));
  FX_INIT_CK(cudaMemset(ctx->b, 0, N * sizeof(double)));
  FX_INIT_CK(cudaMemset(ctx->Pbuf, 0, ctx->ncomp * N * sizeof(double)));
  FX_INIT_CK(cudaMemset(ctx->e_arena, 0, ctx->arena * tsz));
  FX_INIT_CK(cudaMemset(ctx->r_arena, 0, ctx->arena * tsz));
  if (ctx->s_arena) FX_INIT_CK(cudaMemset(ctx->s_arena, 0, ctx->arena * tsz));
  FX_INIT_CK(cudaMemset(ctx->stats_d, 0, sizeof(DevStats)));
  DevParams p0{0.0, 0.0};
  FX_INIT_CK(cudaMemcpy(ctx->params_d, &p0, sizeof(p0), cudaMemcpyHostToDevice));
  FX_INIT_CK(cudaDeviceSynchronize());
  rc = mixed ? build_graphs_t<float>(ctx) : build_graphs_t<double>(ctx);
  if (rc != FERROX_OK && g_pdl) {
    // graph capture without programmatic edges (same kernels, plain dependencies)
    cudaGetLastError();
    for (auto* g : {&ctx->ge_step, &ctx->ge_solve, &ctx->ge_tdgl})
      if (*g) { cudaGraphExecDestroy(*g); *g = nullptr; }
    for (auto* g : {&ctx->gr_step, &ctx->gr_solve, &ctx->gr_tdgl})
      if (*g) { cudaGraphDestroy(*g); *g = nullptr; }
    cudaStreamCaptureStatus cs;
    if (cudaStreamIsCapturing(ctx->cap1, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
      cudaGraph_t junk;
      cudaStreamEndCapture(ctx->cap1, &junk);
      if (junk) cudaGraphDestroy(junk);
    }
    g_pdl = 0;
    rc = mixed ? build_graphs_t<float>(ctx) : build_graphs_t<double>(ctx);
  }
  if (rc != FERROX_OK) return cleanup(rc);
#undef FX_INIT_CK
  *out = ctx;
  return FERROX_OK;
}

ferrox_status ferrox_set_bias(ferrox_ctx* ctx, double v_bottom, double v_top) {
  if (!ctx) return fail(nullptr, FERROX_EINVAL, "null context");
  if (!std::isfinite(v_bottom) || !std::isfinite(v_top)) return fail(ctx, FERROX_EINVAL, "bias not finite");
  ctx->v_bot = v_bottom;
  ctx->v_top = v_top;
  launch_set_params(ctx->params_d, v_bottom, v_top, ctx->stream);
  if (ctx->direct)
    launch_static_b(ctx->b, ctx->planes_d, ctx->params_d, ctx->nx, ctx->ny, ctx->nz, ctx->stream);
  FX_CK(cudaGetLastError());
  return FERROX_OK;
}

ferrox_status ferrox_solve_poisson(ferrox_ctx* ctx) {
  if (!ctx) return fail(nullptr, FERROX_EINVAL, "null context");
  // b of the dynamic planes from the current P, then the converged solve (Step 0)
  launch_tdgl(tdgl_args(ctx, 3), ctx->stream);
  FX_CK(cudaGetLastError());
  FX_CK(cudaGraphLaunch(ctx->ge_solve, ctx->stream));
  if (ctx->num.guess == 1)   // no history yet: the first step starts from this potential
    FX_CK(cudaMemcpyAsync(ctx->phi_prev, ctx->phi, (size_t)ctx->nx * ctx->ny * ctx->nz * sizeof(double),
                          cudaMemcpyDeviceToDevice, ctx->stream));
  return FERROX_OK;
}

ferrox_status ferrox_tdgl_update(ferrox_ctx* ctx) {
  if (!ctx) return fail(nullptr, FERROX_EINVAL, "null context");
  FX_CK(cudaGraphLaunch(ctx->ge_tdgl, ctx->stream));
  return FERROX_OK;
}

ferrox_status ferrox_step(ferrox_ctx* ctx, int nsteps) {
  if (!ctx) return fail(nullptr, FERROX_EINVAL, "null context");
  if (nsteps < 0) return fail(ctx, FERROX_EINVAL, "nsteps < 0");
  for (int q = 0; q < nsteps; ++q) {
    if (ctx->nn_mode == 1) {
      const ferrox_status rc = ctx->num.precision == FERROX_MIXED ? collect_step_t<float>(ctx)
                                                                 : collect_step_t<double>(ctx);
      if (rc != FERROX_OK) return rc;
    } else if (ctx->nn_mode == 2) {
      FX_CK(cudaGraphLaunch(ctx->ge_step_nn, ctx->stream));
    } else {
      FX_CK(cudaGraphLaunch(ctx->ge_step, ctx->stream));
    }
  }
  return FERROX_OK;
}

ferrox_status ferrox_attach_nn(ferrox_ctx* ctx, ferrox_nn* nn, int mode) {
  if (!ctx) return fail(nullptr, FERROX_EINVAL, "null context");
  if (mode < 0 || mode > 2 || (mode > 0 && !nn)) return fail(ctx, FERROX_EINVAL, "bad mode or network");
  FX_CK(cudaStreamSynchronize(ctx->stream));
  if (mode == 0) { ctx->nn_mode = 0; ctx->nn = nullptr; return FERROX_OK; }
  const int l = ctx->nn_level;
  if ((int)ctx->lv.size() <= l) return fail(ctx, FERROX_EINVAL, "the hierarchy has no network level");
  for (int q = 0; q < l; ++q)
    if (!(ctx->lv[q].crx && ctx->lv[q].cry && ctx->lv[q].crz))
      return fail(ctx, FERROX_EINVAL, "the network level must be reached by full 2x2x2 coarsening");
  const NNGrid g = nn_grid(nn);
  const LevelDesc& L = ctx->lv[l];
  if (g.D != L.nz || g.H != L.ny || g.W != L.nx)
    return fail(ctx, FERROX_EINVAL, "network grid does not match the network level of this context");
  if (mode == 1 && nn_capacity(nn) < 1) return fail(ctx, FERROX_EINVAL, "network has no snapshot store");
  if (!ctx->nn_scale) {
    FX_CK(cudaMalloc(&ctx->nn_scale, 2 * sizeof(double)));   // rms of r, ||r|| of the guess
    FX_CK(cudaMalloc(&ctx->phi_guess, (size_t)ctx->nx * ctx->ny * ctx->nz * sizeof(double)));
    FX_CK(cudaMalloc(&ctx->nn_stats, sizeof(DevStats)));
    FX_CK(cudaMemset(ctx->nn_stats, 0, sizeof(DevStats)));
    std::vector<float> pf(4 * L.nz);
    const int fz = ctx->nz / L.nz;
    for (int K = 0; K < L.nz; ++K) {
      double eps = 0.0, fe = 0.0, sc = 0.0;
      for (int k = K * fz; k < (K + 1) * fz; ++k) {
        eps += ctx->epsr[k];
        fe += ctx->planes[k].fe;
        sc += ctx->planes[k].sc;
      }
      pf[4 * K] = (float)(eps / fz / 24.0);
      pf[4 * K + 1] = (float)(fe / fz);
      pf[4 * K + 2] = (float)(sc / fz);
      pf[4 * K + 3] = (float)((K + 0.5) / L.nz);
    }
    FX_CK(cudaMalloc(&ctx->nn_pf, pf.size() * sizeof(float)));
    FX_CK(cudaMemcpy(ctx->nn_pf, pf.data(), pf.size() * sizeof(float), cudaMemcpyHostToDevice));
  }
  ctx->nn = nn;
  ctx->nn_mode = mode;
  if (mode == 2) {
    if (ctx->ge_step_nn) { cudaGraphExecDestroy(ctx->ge_step_nn); ctx->ge_step_nn = nullptr; }
    if (ctx->gr_step_nn) { cudaGraphDestroy(ctx->gr_step_nn); ctx->gr_step_nn = nullptr; }
    const ferrox_status rc = ctx->num.precision == FERROX_MIXED ? build_nn_graph_t<float>(ctx)
                                                               : build_nn_graph_t<double>(ctx);
    if (rc != FERROX_OK) { ctx->nn_mode = 0; return rc; }
  }
  return FERROX_OK;
}

ferrox_status ferrox_profile_step(ferrox_ctx* ctx, double* ms, int* count) {
  return ferrox_profile_step_bytes(ctx, ms, count, nullptr);
}

ferrox_status ferrox_profile_step_bytes(ferrox_ctx* ctx, double* ms, int* count, double* bytes) {
  if (!ctx || !ms || !count) return fail(ctx, FERROX_EINVAL, "null argument");
  return ctx->num.precision == FERROX_MIXED ? profile_step_t<float>(ctx, ms, count, bytes)
                                            : profile_step_t<double>(ctx, ms, count, bytes);
}

ferrox_status ferrox_sync_stats(ferrox_ctx* ctx, ferrox_stats* out) {
  if (!ctx || !out) return fail(ctx, FERROX_EINVAL, "null argument");
  DevStats st{};
  FX_CK(cudaMemcpyAsync(ctx->host_pinned, ctx->stats_d, sizeof(DevStats), cudaMemcpyDeviceToHost,
                        ctx->stream));
  FX_CK(cudaStreamSynchronize(ctx->stream));
  std::memcpy(&st, ctx->host_pinned, sizeof(DevStats));
  out->steps = st.steps;
  out->launches = st.launches;
  out->solves = st.solves;
  out->cycles = st.cycles;
  out->vcycles = st.vcycles;
  out->nn_rejected = st.nn_rejected;
  out->last_cycles = st.last_cycles;
  out->last_rel_res = st.last_rel;
  out->status = st.status;
  if (st.status != FERROX_OK) {
    ctx->err = st.status == FERROX_ENOCONV ? "Poisson solve reached max_cycles above tolerance"
               : st.status == FERROX_ENONFINITE ? "non-finite residual norm"
                                                : "device status set";
    return (ferrox_status)st.status;
  }
  return FERROX_OK;
}

ferrox_status ferrox_clear_status(ferrox_ctx* ctx) {
  if (!ctx) return fail(nullptr, FERROX_EINVAL, "null context");
  // status is the 5th field group; clear it with a small async copy of zero
  static const int zero = 0;
  FX_CK(cudaMemcpyAsync(reinterpret_cast<char*>(ctx->stats_d) + offsetof(DevStats, status), &zero,
                        sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
  FX_CK(cudaStreamSynchronize(ctx->stream));
  return FERROX_OK;
}

ferrox_status ferrox_charge(ferrox_ctx* ctx, ferrox_charge_t* out) {
  if (!ctx || !out) return fail(ctx, FERROX_EINVAL, "null argument");
  ChargeArgs a{};
  const long long N = (long long)ctx->nx * ctx->ny * ctx->nz;
  a.phi = ctx->phi;
  a.P = ctx->P + (long long)(ctx->ncomp - 1) * N;
  a.planes = ctx->planes_d;
  a.params = ctx->params_d;
  a.nx = ctx->nx; a.ny = ctx->ny; a.nz = ctx->nz; a.k_int = ctx->k_int;
  a.h = ctx->h; a.eps0 = kEps0;
  a.eps_top = kEps0 * ctx->epsr[ctx->nz - 1];
  a.eps_bot = kEps0 * ctx->epsr[0];
  a.eps_L = ctx->k_int > 0 ? kEps0 * ctx->epsr[ctx->k_int - 1] : 0.0;
  a.eps_R = kEps0 * ctx->epsr[ctx->k_int];
  a.out = ctx->charge_d;
  a.partials = ctx->charge_part_d;
  launch_charge(a, ctx->stream);
  FX_CK(cudaGetLastError());
  FX_CK(cudaMemcpyAsync(ctx->host_pinned, ctx->charge_d, 4 * sizeof(double), cudaMemcpyDeviceToHost,
                        ctx->stream));
  FX_CK(cudaStreamSynchronize(ctx->stream));
  const double inv = 1.0 / ((double)ctx->nx * ctx->ny);
  const double* s = ctx->host_pinned;
  out->Q_int = -s[0] * inv;
  out->phi_int_avg = s[1] * inv;
  out->V_fe = ctx->v_top - out->phi_int_avg;
  out->sigma_top = -s[2] * inv;
  out->sigma_bot = s[3] * inv;
  ferrox_stats st;
  return ferrox_sync_stats(ctx, &st);
}

ferrox_status ferrox_residual(ferrox_ctx* ctx, int arithmetic, double* r_host) {
  if (!ctx) return fail(nullptr, FERROX_EINVAL, "null context");
  if (!r_host) return fail(ctx, FERROX_EINVAL, "null output array");
  if (arithmetic != FERROX_RESID_FP64 && arithmetic != FERROX_RESID_DOUBLE_FLOAT)
    return fail(ctx, FERROX_EINVAL, "arithmetic must be FERROX_RESID_FP64 or FERROX_RESID_DOUBLE_FLOAT");
  cudaStream_t s = ctx->stream;
  const long long N = (long long)ctx->nx * ctx->ny * ctx->nz;
  double* r_d = nullptr;
  FX_CK(cudaMalloc(&r_d, N * sizeof(double)));
  // the right-hand side of the current polarization, then r = b + rho(phi) - A phi
  launch_tdgl(tdgl_args(ctx, 3), s);
  ResidArgs a{};
  a.phi = ctx->phi; a.b = ctx->b; a.planes = ctx->planes_d; a.coef0 = ctx->coef0;
  a.params = ctx->params_d;
  a.nx = ctx->nx; a.ny = ctx->ny; a.nz = ctx->nz;
  a.r_out = r_d;
  a.s_out = nullptr;
  a.carriers = carrier_kind(ctx);
  a.coef_df = arithmetic == FERROX_RESID_DOUBLE_FLOAT ? ctx->coef_df : nullptr;
  a.kchunk = arithmetic == FERROX_RESID_DOUBLE_FLOAT ? ctx->resid_kchunk_df : ctx->resid_kchunk;
  a.no_stats = 1;
  a.stats = ctx->stats_d;
  a.partials = ctx->partials_d;
  launch_resid<double>(a, s);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(r_host, r_d, N * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(r_d);
  if (e != cudaSuccess) return fail(ctx, FERROX_ECUDA, std::string("ferrox_residual: ") + cudaGetErrorString(e));
  return FERROX_OK;
}

ferrox_status ferrox_qv_sweep(ferrox_ctx* ctx, const double* v_app, int npoints, int steps_per_point,
                              ferrox_charge_t* out) {
  if (!ctx) return fail(nullptr, FERROX_EINVAL, "null context");
  if (!v_app || !out || npoints < 1 || steps_per_point < 0)
    return fail(ctx, FERROX_EINVAL, "ferrox_qv_sweep: need bias and output arrays, npoints >= 1, "
                                    "steps_per_point >= 0");
  for (int q = 0; q < npoints; ++q) {
    ferrox_status rc = ferrox_set_bias(ctx, 0.0, v_app[q]);
    if (rc == FERROX_OK && steps_per_point > 0) rc = ferrox_step(ctx, steps_per_point);
    if (rc == FERROX_OK) rc = ferrox_charge(ctx, &out[q]);
    if (rc != FERROX_OK) return rc;
  }
  return FERROX_OK;
}

ferrox_status ferrox_get_state(ferrox_ctx* ctx, double* P_host, double* phi_host) {
  if (!ctx) return fail(nullptr, FERROX_EINVAL, "null context");
  const long long N = (long long)ctx->nx * ctx->ny * ctx->nz;
  if (P_host)
    FX_CK(cudaMemcpyAsync(P_host, ctx->P, ctx->ncomp * N * sizeof(double), cudaMemcpyDeviceToHost,
                          ctx->stream));
  if (phi_host)
    FX_CK(cudaMemcpyAsync(phi_host, ctx->phi, N * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  ferrox_stats st;
  return ferrox_sync_stats(ctx, &st);
}

ferrox_status ferrox_set_state(ferrox_ctx* ctx, const double* P_host, const double* phi_host) {
  if (!ctx) return fail(nullptr, FERROX_EINVAL, "null context");
  const long long N = (long long)ctx->nx * ctx->ny * ctx->nz;
  if (P_host)
    FX_CK(cudaMemcpyAsync(ctx->P, P_host, ctx->ncomp * N * sizeof(double), cudaMemcpyHostToDevice,
                          ctx->stream));
  if (phi_host) {
    FX_CK(cudaMemcpyAsync(ctx->phi, phi_host, N * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    if (ctx->num.guess == 1)   // a new state has no history
      FX_CK(cudaMemcpyAsync(ctx->phi_prev, ctx->phi, N * sizeof(double), cudaMemcpyDeviceToDevice,
                            ctx->stream));
  }
  return FERROX_OK;
}

ferrox_status ferrox_fe_planes(const ferrox_ctx* ctx, int* fe_lo, int* fe_hi) {
  if (!ctx || !fe_lo || !fe_hi) return FERROX_EINVAL;
  *fe_lo = ctx->fe_lo;
  *fe_hi = ctx->fe_hi;
  return FERROX_OK;
}

ferrox_status ferrox_get_state_fe(ferrox_ctx* ctx, double* P_fe_host, double* phi_host) {
  if (!ctx) return fail(nullptr, FERROX_EINVAL, "null context");
  const long long plane = (long long)ctx->nx * ctx->ny, N = plane * ctx->nz;
  const long long nfe = (long long)(ctx->fe_hi - ctx->fe_lo + 1) * plane;
  if (P_fe_host)
    for (int q = 0; q < ctx->ncomp; ++q)
      FX_CK(cudaMemcpyAsync(P_fe_host + q * nfe, ctx->P + q * N + ctx->fe_lo * plane,
                            nfe * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  if (phi_host)
    FX_CK(cudaMemcpyAsync(phi_host, ctx->phi, N * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  ferrox_stats st;
  return ferrox_sync_stats(ctx, &st);
}

ferrox_status ferrox_set_state_fe(ferrox_ctx* ctx, const double* P_fe_host, const double* phi_host) {
  if (!ctx) return fail(nullptr, FERROX_EINVAL, "null context");
  const long long plane = (long long)ctx->nx * ctx->ny, N = plane * ctx->nz;
  const long long nfe = (long long)(ctx->fe_hi - ctx->fe_lo + 1) * plane;
  if (P_fe_host)
    for (int q = 0; q < ctx->ncomp; ++q)
      FX_CK(cudaMemcpyAsync(ctx->P + q * N + ctx->fe_lo * plane, P_fe_host + q * nfe,
                            nfe * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  if (phi_host) {
    FX_CK(cudaMemcpyAsync(ctx->phi, phi_host, N * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    if (ctx->num.guess == 1)   // a new state has no history
      FX_CK(cudaMemcpyAsync(ctx->phi_prev, ctx->phi, N * sizeof(double), cudaMemcpyDeviceToDevice,
                            ctx->stream));
  }
  return FERROX_OK;
}

ferrox_status ferrox_destroy(ferrox_ctx* ctx) {
  release(ctx);
  return FERROX_OK;
}

const char* ferrox_last_error(const ferrox_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_init_error.c_str();
}

ferrox_status ferrox_level_shape(const ferrox_ctx* ctx, int l, int* nx, int* ny, int* nz,
                                 int* nlevels) {
  if (!ctx) return FERROX_EINVAL;
  if (nlevels) *nlevels = (int)ctx->lv.size();
  if (l < 0 || l >= (int)ctx->lv.size()) return FERROX_EINVAL;
  if (nx) *nx = ctx->lv[l].nx;
  if (ny) *ny = ctx->lv[l].ny;
  if (nz) *nz = ctx->lv[l].nz;
  return FERROX_OK;
}

}  // extern "C"


// ---- batched persistent engine (host side) ---------------------------------------------
//
// n independent MFIM/MFISM instances (uneven lateral sizes, own biases) packed
// back to back in the caller's P and phi arrays; one cooperative launch runs
// whole time steps of all of them (persistent.cu).  The launch shape (threads
// per block, rows per work unit) is chosen by timing the candidates on the
// first step, on a saved copy of the state, and cached per problem shape.

struct BatchPlan {     // one instance, planned with the single-instance machinery
  ferrox_ctx c;
  long long cell_off = 0, arena_off = 0;
  int coef_off = 0, coef0_off = 0, plane_off = 0, lv_off = 0, lvt_off = 0;
};

struct ferrox_batch {
  int n = 0;
  ferrox_numerics num{};
  bool mixed = false;
  size_t tsz = 8;
  cudaStream_t stream = nullptr, cap = nullptr;
  std::vector<BatchPlan> plans;
  long long cells = 0, arena = 0;
  int Ldown = 0, any_full_tail = 0, nrows = 0;
  double* P = nullptr;
  double* phi = nullptr;
  double* b = nullptr;
  double* Pbuf = nullptr;
  double* backup = nullptr;
  void* e = nullptr;
  void* r = nullptr;
  void* s = nullptr;
  void* coef = nullptr;
  void* dense = nullptr;              // T: inverses of the instances' dense tail levels
  PlaneCoef<double>* coef0 = nullptr;
  PlaneTDGL* planes = nullptr;
  LevelDesc* lv = nullptr;
  LevelDesc* lvt = nullptr;
  int* pre = nullptr;
  double* partials = nullptr;
  int* active = nullptr;
  GridBar* bar = nullptr;             // one per CTA group (n at most)
  int* grp_d = nullptr;               // CTA prefix [n+1], then instance prefix [n+1]
  int ngroups = 1;
  bool grouped = false;
  int* status = nullptr;
  unsigned int* ticket = nullptr;     // decision kernel of the graph engine: blocks done
  int* tile_pre = nullptr;            // graph engine's TDGL: prefix of column tiles per instance
  int* any_d = nullptr;               // phase profile: "any instance active" (device / pinned host)
  int* any_h = nullptr;
  int ntiles = 0;
  int* nsteps_d = nullptr;
  int* dbg = nullptr;
  DevParams* params = nullptr;
  DevStats* stats = nullptr;
  BatchInst* inst = nullptr;
  double* charge_part = nullptr;
  double* charge_out = nullptr;
  double* host_pinned = nullptr;
  int threads = 512, rows_per_unit = 1, blocks = 0;
  size_t smem = 0;
  bool tuned = false;
  int engine = 0;                     // 0: one persistent launch; 1: a graph of per-phase launches
  int unit_blocks = 0;                // CTAs of the per-phase launches (engine 1)
  cudaStream_t cap2 = nullptr;        // captures the phase graph's WHILE body
  cudaGraphExec_t ge_step = nullptr, ge_solve = nullptr;
  cudaGraph_t gr_step = nullptr, gr_solve = nullptr;
  std::string err;
};

namespace {

std::mutex g_tune_mu;
struct TuneChoice { int threads, rows, bps, grouped, engine; };
std::vector<std::pair<std::string, TuneChoice>> g_tune_cache;

ferrox_status bfail(ferrox_batch* b, ferrox_status s, const std::string& m) {
  if (b) b->err = m; else g_init_error = m;
  return s;
}

#define FX_BCK(call)                                                                          \
  do {                                                                                        \
    cudaError_t _e = (call);                                                                  \
    if (_e != cudaSuccess)                                                                    \
      return bfail(B, _e == cudaErrorMemoryAllocation ? FERROX_ENOMEM : FERROX_ECUDA,         \
                   std::string(#call) + ": " + cudaGetErrorString(_e));                       \
  } while (0)

std::vector<int> batch_prefix(const ferrox_batch* B, int R) {
  const int n = B->n, L = B->Ldown;
  std::vector<int> pre((size_t)(1 + 2 * L) * (n + 1), 0);
  for (int i = 0; i < n; ++i) pre[i + 1] = pre[i] + B->plans[i].c.ny;
  for (int l = 0; l < L; ++l) {
    int* ps = &pre[(size_t)(1 + l) * (n + 1)];
    int* pc = &pre[(size_t)(1 + L + l) * (n + 1)];
    for (int i = 0; i < n; ++i) {
      const ferrox_ctx& c = B->plans[i].c;
      int us = 0, uc = 0;
      if (l < c.tail_first) {
        const LevelDesc& F = c.lv[l];
        const LevelDesc& C = c.lv[l + 1];
        us = F.nz * ((F.ny + R - 1) / R);
        uc = C.nz * ((C.ny + R - 1) / R);
      }
      ps[i + 1] = ps[i] + us;
      pc[i + 1] = pc[i] + uc;
    }
  }
  return pre;
}

BatchArgs batch_args(ferrox_batch* B, int mode) {
  BatchArgs a{};
  a.inst = B->inst; a.ninst = B->n; a.mode = mode; a.nsteps = B->nsteps_d;
  a.e = B->e; a.r = B->r; a.s = B->s; a.coef = B->coef; a.lv = B->lv; a.lvt = B->lvt;
  a.dense = B->dense;
  a.pre = B->pre; a.Ldown = B->Ldown; a.partials = B->partials; a.active = B->active;
  a.bar = B->bar; a.status = B->status; a.tol = B->num.tol; a.max_cycles = B->num.max_cycles;
  a.grp_cta = B->grp_d; a.grp_inst = B->grp_d + (B->n + 1); a.ngroups = B->ngroups;
  a.nu1 = B->num.nu1; a.nu2 = B->num.nu2; a.rows_per_unit = B->rows_per_unit;
  a.any_full_tail = B->any_full_tail;
  a.dbg = B->dbg;
  a.ticket = B->ticket;
  a.tile_pre = B->tile_pre;
  a.ntiles = B->ntiles;
  return a;
}

cudaError_t batch_launch(ferrox_batch* B, int mode, cudaStream_t s) {
  const BatchArgs a = batch_args(B, mode);
  return B->mixed ? launch_batch<float>(a, B->blocks, B->threads, B->smem, s)
                  : launch_batch<double>(a, B->blocks, B->threads, B->smem, s);
}

// CTA groups.  grouped = false: one group, every CTA and instance.  grouped =
// true: contiguous instance ranges of about cells / blocks cells each, and CTAs
// shared out in proportion to their cells (at least one each), so instances of
// different groups advance without waiting for each other at a barrier.
void batch_groups(const ferrox_batch* B, int blocks, bool grouped, std::vector<int>& gcta,
                  std::vector<int>& ginst) {
  const int n = B->n;
  gcta.assign(1, 0);
  ginst.assign(1, 0);
  if (!grouped || blocks < 2) {
    gcta.push_back(blocks);
    ginst.push_back(n);
    return;
  }
  long long total = 0;
  std::vector<long long> cells(n);
  for (int i = 0; i < n; ++i) {
    const ferrox_ctx& c = B->plans[i].c;
    cells[i] = (long long)c.nx * c.ny * c.nz;
    total += cells[i];
  }
  const double target = (double)total / blocks;
  std::vector<long long> gcells;
  long long acc = 0;
  for (int i = 0; i < n; ++i) {
    acc += cells[i];
    if (acc >= target || i == n - 1) {
      ginst.push_back(i + 1);
      gcells.push_back(acc);
      acc = 0;
    }
  }
  while ((int)gcells.size() > blocks) {   // merge the last two groups
    gcells[gcells.size() - 2] += gcells.back();
    gcells.pop_back();
    ginst.erase(ginst.end() - 2);
  }
  const int G = (int)gcells.size();
  std::vector<int> k(G, 1);
  std::vector<double> rem(G);
  int left = blocks - G;
  for (int q = 0; q < G; ++q) {
    const double quota = (double)gcells[q] / total * blocks;
    const int extra = std::max(0, std::min(left, (int)quota - 1));
    k[q] += extra;
    left -= extra;
    rem[q] = quota - k[q];
  }
  while (left > 0) {   // largest remainder
    int best = 0;
    for (int q = 1; q < G; ++q) if (rem[q] > rem[best]) best = q;
    k[best] += 1;
    rem[best] -= 1.0;
    --left;
  }
  for (int q = 0; q < G; ++q) gcta.push_back(gcta.back() + k[q]);
}

ferrox_status batch_configure(ferrox_batch* B, int threads, int R, int bps = 1, int grouped = 0) {
  int per_sm = 0;
  FX_BCK(B->mixed ? batch_occupancy<float>(threads, B->smem, &per_sm)
                  : batch_occupancy<double>(threads, B->smem, &per_sm));
  if (per_sm < 1) return bfail(B, FERROX_ECUDA, "batch kernel does not fit on an SM");
  int dev = 0, sms = 0;
  FX_BCK(cudaGetDevice(&dev));
  FX_BCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  B->threads = threads;
  B->rows_per_unit = R;
  // bps CTAs per SM, never more than the occupancy calculation allows (the
  // cooperative launch then guarantees they are all resident together)
  B->blocks = sms * std::min(bps, per_sm);
  const std::vector<int> pre = batch_prefix(B, R);
  FX_BCK(cudaMemcpy(B->pre, pre.data(), pre.size() * sizeof(int), cudaMemcpyHostToDevice));
  std::vector<int> gcta, ginst;
  batch_groups(B, B->blocks, grouped != 0, gcta, ginst);
  B->grouped = grouped != 0;
  B->ngroups = (int)gcta.size() - 1;
  std::vector<int> g(2 * (B->n + 1), 0);
  std::copy(gcta.begin(), gcta.end(), g.begin());
  std::copy(ginst.begin(), ginst.end(), g.begin() + (B->n + 1));
  FX_BCK(cudaMemcpy(B->grp_d, g.data(), g.size() * sizeof(int), cudaMemcpyHostToDevice));
  return FERROX_OK;
}

std::string batch_key(const ferrox_batch* B) {
  std::string k = B->mixed ? "f32" : "f64";
  for (const auto& p : B->plans)
    k += ":" + std::to_string(p.c.nx) + "x" + std::to_string(p.c.ny) + "x" + std::to_string(p.c.nz);
  return k;
}

// the graph of per-phase launches of one step (mode 0) or one solve (mode 1)
ferrox_status phase_graph(ferrox_batch* B, int mode, cudaGraph_t* g, cudaGraphExec_t* ge) {
  *g = nullptr;
  *ge = nullptr;
  const BatchArgs a = batch_args(B, mode);
  FX_BCK(cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeRelaxed));
  const cudaError_t le = B->mixed ? capture_phases<float>(a, B->unit_blocks, B->smem, B->cap, B->cap2)
                                  : capture_phases<double>(a, B->unit_blocks, B->smem, B->cap, B->cap2);
  const cudaError_t ce = cudaStreamEndCapture(B->cap, g);
  if (le != cudaSuccess || ce != cudaSuccess) {
    if (*g) cudaGraphDestroy(*g);
    *g = nullptr;
    cudaGetLastError();
    return bfail(B, FERROX_ECUDA, std::string("capturing the phase graph: ") +
                                      cudaGetErrorString(le != cudaSuccess ? le : ce));
  }
  FX_BCK(cudaGraphInstantiate(ge, *g, 0));
  return FERROX_OK;
}

// the per-phase launches: one-row units, eight CTAs of 256 threads per SM
ferrox_status phase_configure(ferrox_batch* B, int R = 1) {
  int dev = 0, sms = 0;
  FX_BCK(cudaGetDevice(&dev));
  FX_BCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const ferrox_status rc = batch_configure(B, 256, R, 1, 0);
  if (rc != FERROX_OK) return rc;
  B->unit_blocks = 8 * sms;
  return FERROX_OK;
}

// time each candidate launch shape on one step from a saved state, keep the fastest;
// the candidates are the persistent kernel's shapes and the graph of per-phase launches
ferrox_status batch_autotune(ferrox_batch* B) {
  const std::string key = batch_key(B);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (auto& kv : g_tune_cache)
      if (kv.first == key) {
        B->engine = kv.second.engine;
        if (B->engine == 1) return phase_configure(B, kv.second.rows);
        return batch_configure(B, kv.second.threads, kv.second.rows, kv.second.bps, kv.second.grouped);
      }
  }
  const size_t bytes = (size_t)B->cells * sizeof(double);
  cudaStream_t s = B->stream;
  FX_BCK(cudaMemcpyAsync(B->backup, B->P, bytes, cudaMemcpyDeviceToDevice, s));
  FX_BCK(cudaMemcpyAsync(B->backup + B->cells, B->phi, bytes, cudaMemcpyDeviceToDevice, s));
  std::vector<DevStats> st0(B->n);
  FX_BCK(cudaMemcpyAsync(st0.data(), B->stats, B->n * sizeof(DevStats), cudaMemcpyDeviceToHost, s));
  FX_BCK(cudaStreamSynchronize(s));
  const int one = 1;
  FX_BCK(cudaMemcpy(B->nsteps_d, &one, sizeof(int), cudaMemcpyHostToDevice));
  cudaEvent_t e0, e1;
  FX_BCK(cudaEventCreate(&e0));
  FX_BCK(cudaEventCreate(&e1));
  float best = 1e30f;
  int bt = 512, bR = 1, bB = 1, bG = 0;
  const int cand_t[2] = {256, 512}, cand_R[3] = {1, 2, 4}, cand_b[2] = {1, 2};
  for (int gi = 0; gi < 2; ++gi)
  for (int bi = 0; bi < 2; ++bi)
  for (int ti = 0; ti < 2; ++ti)
    for (int ri = 0; ri < 3; ++ri) {
      int per_sm = 0;
      FX_BCK(B->mixed ? batch_occupancy<float>(cand_t[ti], B->smem, &per_sm)
                      : batch_occupancy<double>(cand_t[ti], B->smem, &per_sm));
      if (cand_b[bi] > per_sm) continue;
      ferrox_status rc = batch_configure(B, cand_t[ti], cand_R[ri], cand_b[bi], gi);
      if (rc != FERROX_OK) return rc;
      FX_BCK(cudaEventRecord(e0, s));
      FX_BCK(batch_launch(B, 0, s));
      FX_BCK(cudaEventRecord(e1, s));
      FX_BCK(cudaEventSynchronize(e1));
      float ms = 0.f;
      FX_BCK(cudaEventElapsedTime(&ms, e0, e1));
      int gst = 0;
      FX_BCK(cudaMemcpy(&gst, B->status, sizeof(int), cudaMemcpyDeviceToHost));
      if (gst != 0) return bfail(B, (ferrox_status)gst, "batch kernel failed while tuning");
      if (ms < best) { best = ms; bt = cand_t[ti]; bR = cand_R[ri]; bB = cand_b[bi]; bG = gi; }
      FX_BCK(cudaMemcpyAsync(B->P, B->backup, bytes, cudaMemcpyDeviceToDevice, s));
      FX_BCK(cudaMemcpyAsync(B->phi, B->backup + B->cells, bytes, cudaMemcpyDeviceToDevice, s));
      FX_BCK(cudaMemcpyAsync(B->stats, st0.data(), B->n * sizeof(DevStats), cudaMemcpyHostToDevice, s));
      FX_BCK(cudaStreamSynchronize(s));
    }
  // the graph of per-phase launches with 1, 2 or 4 rows per work unit: the
  // better of two launches each (the first uploads the graph)
  int engine = 0, pR = 1;
  for (int ri = 0; ri < 3; ++ri) {
    ferrox_status rc = phase_configure(B, cand_R[ri]);
    if (rc != FERROX_OK) return rc;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    rc = phase_graph(B, 0, &g, &ge);
    if (rc != FERROX_OK) return rc;
    float pbest = 1e30f;
    for (int rep = 0; rep < 2 && rc == FERROX_OK; ++rep) {
      cudaError_t e = cudaEventRecord(e0, s);
      if (e == cudaSuccess) e = cudaGraphLaunch(ge, s);
      if (e == cudaSuccess) e = cudaEventRecord(e1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      int gst = 0;
      if (e == cudaSuccess) e = cudaMemcpy(&gst, B->status, sizeof(int), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) rc = bfail(B, FERROX_ECUDA, cudaGetErrorString(e));
      else if (gst != 0) rc = bfail(B, (ferrox_status)gst, "phase graph failed while tuning");
      pbest = std::min(pbest, ms);
      if (rc == FERROX_OK) {
        e = cudaMemcpyAsync(B->P, B->backup, bytes, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(B->phi, B->backup + B->cells, bytes, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(B->stats, st0.data(), B->n * sizeof(DevStats), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = bfail(B, FERROX_ECUDA, cudaGetErrorString(e));
      }
    }
    cudaGraphExecDestroy(ge);
    cudaGraphDestroy(g);
    if (rc != FERROX_OK) return rc;
    if (pbest < best) { best = pbest; engine = 1; pR = cand_R[ri]; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache.push_back({key, {bt, engine == 1 ? pR : bR, bB, bG, engine}});
  }
  B->engine = engine;
  if (engine == 1) return phase_configure(B, pR);
  return batch_configure(B, bt, bR, bB, bG);
}

ferrox_status batch_build_graphs(ferrox_batch* B) {
  if (B->engine == 1) {
    ferrox_status rc = phase_graph(B, 0, &B->gr_step, &B->ge_step);
    if (rc == FERROX_OK) rc = phase_graph(B, 1, &B->gr_solve, &B->ge_solve);
    return rc;
  }
  for (int mode = 0; mode < 2; ++mode) {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    FX_BCK(cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeRelaxed));
    cudaError_t le = batch_launch(B, mode, B->cap);
    cudaError_t ce = cudaStreamEndCapture(B->cap, &g);
    if (le != cudaSuccess || ce != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return bfail(B, FERROX_ECUDA, std::string("capturing the batch launch: ") +
                                        cudaGetErrorString(le != cudaSuccess ? le : ce));
    }
    FX_BCK(cudaGraphInstantiate(&ge, g, 0));
    if (mode == 0) { B->gr_step = g; B->ge_step = ge; } else { B->gr_solve = g; B->ge_solve = ge; }
  }
  return FERROX_OK;
}

void batch_release(ferrox_batch* B) {
  if (!B) return;
  if (B->stream) cudaStreamSynchronize(B->stream);
  if (B->ge_step) cudaGraphExecDestroy(B->ge_step);
  if (B->ge_solve) cudaGraphExecDestroy(B->ge_solve);
  if (B->gr_step) cudaGraphDestroy(B->gr_step);
  if (B->gr_solve) cudaGraphDestroy(B->gr_solve);
  void* ptrs[] = {B->b, B->Pbuf, B->backup, B->e, B->r, B->s, B->coef, B->dense, B->coef0, B->planes, B->lv,
                  B->lvt, B->pre, B->partials, B->active, B->bar, B->grp_d, B->status, B->ticket, B->tile_pre, B->any_d, B->nsteps_d, B->dbg, B->params,
                  B->stats, B->inst, B->charge_part, B->charge_out};
  for (void* p : ptrs) if (p) cudaFree(p);
  if (B->host_pinned) cudaFreeHost(B->host_pinned);
  if (B->any_h) cudaFreeHost(B->any_h);
  if (B->cap) cudaStreamDestroy(B->cap);
  if (B->cap2) cudaStreamDestroy(B->cap2);
  delete B;
}

}  // namespace

extern "C" {

ferrox_status ferrox_init_batch(ferrox_batch** out, int n, const ferrox_geometry* geoms,
                                const ferrox_numerics* num, double* P_dev, double* phi_dev,
                                void* cuda_stream) {
  if (!out) return bfail(nullptr, FERROX_EINVAL, "null output pointer");
  *out = nullptr;
  if (n < 1 || !geoms) return bfail(nullptr, FERROX_EINVAL, "need n >= 1 instances");
  for (int i = 0; i < n; ++i) {
    ferrox_status rc = validate(&geoms[i], num, P_dev, phi_dev);
    if (rc != FERROX_OK) return rc;
    if (geoms[i].ncomp != 1) return bfail(nullptr, FERROX_EINVAL, "batched instances are uniaxial (ncomp = 1)");
  }
  if (num->order != 1) return bfail(nullptr, FERROX_EINVAL, "the batched engine runs order-1 steps");
  if (num->nonlinear != FERROX_NEWTON)
    return bfail(nullptr, FERROX_EINVAL, "the batched engine iterates the carrier charge by Newton");
  if (num->tdgl_arith != FERROX_TDGL_FP64)
    return bfail(nullptr, FERROX_EINVAL, "the batched engine evaluates the TDGL force in FP64");
  if (num->inner > 1 || num->inner < 0)
    return bfail(nullptr, FERROX_EINVAL, "the batched engine runs one V-cycle per outer iteration");
  ferrox_batch* B = new ferrox_batch();
  B->n = n;
  B->num = *num;
  B->mixed = num->precision == FERROX_MIXED;
  B->tsz = B->mixed ? sizeof(float) : sizeof(double);
  B->stream = static_cast<cudaStream_t>(cuda_stream);
  B->P = P_dev;
  B->phi = phi_dev;
  B->plans.resize(n);
  // plan every instance with the single-instance machinery, then pack
  long long cells = 0, arena = 0;
  int ncoef = 0, nplanes = 0, nlv = 0, nlvt = 0;
  size_t smem = 16;
  for (int i = 0; i < n; ++i) {
    BatchPlan& p = B->plans[i];
    ferrox_ctx& c = p.c;
    const ferrox_geometry& g = geoms[i];
    c.nx = g.nx; c.ny = g.ny; c.h = g.h; c.pbc = g.pbc; c.lambda = g.lambda; c.ncomp = 1;
    c.layers.assign(g.layers, g.layers + g.nlayers);
    c.nz = 0;
    for (auto& L : c.layers) c.nz += L.ncells;
    c.num = *num;
    if (build_planes(&c) != FERROX_OK) {
      const std::string m = g_init_error;
      batch_release(B);
      return bfail(nullptr, FERROX_EINVAL, m);
    }
    c.shift = c.has_sc;   // the batched engine iterates by damped Newton
    build_levels(&c);
    plan_tail(&c, B->tsz);
    p.cell_off = cells;
    p.arena_off = arena;
    p.coef_off = ncoef;
    p.coef0_off = nplanes;
    p.plane_off = nplanes;
    p.lv_off = nlv;
    p.lvt_off = nlvt;
    cells += (long long)c.nx * c.ny * c.nz;
    arena += c.arena;
    for (auto& l : c.lv) ncoef += l.nz;
    nplanes += c.nz;
    nlv += (int)c.lv.size();
    nlvt += (int)c.lv_tail.size();
    smem = std::max(smem, c.tail_smem);
    B->Ldown = std::max(B->Ldown, c.tail_first);
    if (c.tail_first == 0) B->any_full_tail = 1;
    B->nrows += c.ny;
  }
  B->cells = cells;
  B->arena = arena;
  if (arena >= (1LL << 31)) {
    batch_release(B);
    return bfail(nullptr, FERROX_EINVAL, "batch too large: the multigrid arenas exceed 2^31 elements");
  }
  // with any semiconductor instance every tail carries the shift array too
  const bool any_sc = std::any_of(B->plans.begin(), B->plans.end(), [](const BatchPlan& p) { return p.c.has_sc; });
  for (const auto& p : B->plans)
    smem = std::max(smem, (size_t)p.c.tail_elems * B->tsz * (any_sc ? 3 : 2));
  B->smem = smem;
  auto cleanup = [&](ferrox_status st) { g_init_error = B->err; batch_release(B); return st; };
#define FX_BINIT(call)                                                                        \
  do {                                                                                        \
    cudaError_t _e = (call);                                                                  \
    if (_e != cudaSuccess) {                                                                  \
      B->err = std::string(#call) + ": " + cudaGetErrorString(_e);                           \
      return cleanup(_e == cudaErrorMemoryAllocation ? FERROX_ENOMEM : FERROX_ECUDA);         \
    }                                                                                         \
  } while (0)
  const size_t tsz = B->tsz;
  const bool has_sc = std::any_of(B->plans.begin(), B->plans.end(), [](const BatchPlan& p) { return p.c.has_sc; });
  FX_BINIT(cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking));
  FX_BINIT(cudaStreamCreateWithFlags(&B->cap2, cudaStreamNonBlocking));
  FX_BINIT(cudaMalloc(&B->b, cells * sizeof(double)));
  FX_BINIT(cudaMalloc(&B->Pbuf, cells * sizeof(double)));
  FX_BINIT(cudaMalloc(&B->backup, 2 * cells * sizeof(double)));
  FX_BINIT(cudaMalloc(&B->e, arena * tsz));
  FX_BINIT(cudaMalloc(&B->r, arena * tsz));
  if (has_sc) FX_BINIT(cudaMalloc(&B->s, arena * tsz));
  FX_BINIT(cudaMalloc(&B->coef, (size_t)ncoef * (B->mixed ? sizeof(PlaneCoef<float>) : sizeof(PlaneCoef<double>))));
  FX_BINIT(cudaMalloc(&B->coef0, (size_t)nplanes * sizeof(PlaneCoef<double>)));
  FX_BINIT(cudaMalloc(&B->planes, (size_t)nplanes * sizeof(PlaneTDGL)));
  FX_BINIT(cudaMalloc(&B->lv, (size_t)nlv * sizeof(LevelDesc)));
  FX_BINIT(cudaMalloc(&B->lvt, (size_t)nlvt * sizeof(LevelDesc)));
  FX_BINIT(cudaMalloc(&B->pre, (size_t)(1 + 2 * B->Ldown) * (n + 1) * sizeof(int)));
  FX_BINIT(cudaMalloc(&B->partials, (size_t)3 * B->nrows * sizeof(double)));
  FX_BINIT(cudaMalloc(&B->active, n * sizeof(int)));
  FX_BINIT(cudaMalloc(&B->bar, (size_t)n * sizeof(GridBar)));
  FX_BINIT(cudaMalloc(&B->grp_d, 2 * (size_t)(n + 1) * sizeof(int)));
  FX_BINIT(cudaMalloc(&B->status, sizeof(int)));
  FX_BINIT(cudaMalloc(&B->ticket, sizeof(unsigned int)));
  FX_BINIT(cudaMalloc(&B->any_d, sizeof(int)));
  FX_BINIT(cudaMallocHost(&B->any_h, sizeof(int)));
  FX_BINIT(cudaMemset(B->ticket, 0, sizeof(unsigned int)));
  {
    std::vector<int> tp(n + 1, 0);
    for (int i = 0; i < n; ++i) {
      const ferrox_ctx& c = B->plans[i].c;
      tp[i + 1] = tp[i] + ((c.nx + kTdglTileX - 1) / kTdglTileX) * ((c.ny + kTdglTileY - 1) / kTdglTileY);
    }
    B->ntiles = tp[n];
    FX_BINIT(cudaMalloc(&B->tile_pre, (n + 1) * sizeof(int)));
    FX_BINIT(cudaMemcpy(B->tile_pre, tp.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice));
  }
  FX_BINIT(cudaMalloc(&B->nsteps_d, sizeof(int)));
  FX_BINIT(cudaMalloc(&B->dbg, (8 + 1024) * sizeof(int)));
  FX_BINIT(cudaMemset(B->dbg, 0, (8 + 1024) * sizeof(int)));
  FX_BINIT(cudaMalloc(&B->params, n * sizeof(DevParams)));
  FX_BINIT(cudaMalloc(&B->stats, n * sizeof(DevStats)));
  FX_BINIT(cudaMalloc(&B->inst, n * sizeof(BatchInst)));
  FX_BINIT(cudaMalloc(&B->charge_part, (size_t)n * 4 * 64 * sizeof(double)));
  FX_BINIT(cudaMalloc(&B->charge_out, (size_t)n * 8 * sizeof(double)));
  FX_BINIT(cudaMallocHost(&B->host_pinned, (size_t)n * 8 * sizeof(double) + 64));
  // tables
  std::vector<unsigned char> coefT, denseT;
  std::vector<PlaneCoef<double>> coef0;
  std::vector<PlaneTDGL> planes;
  std::vector<LevelDesc> lv, lvt;
  std::vector<BatchInst> inst(n);
  for (int i = 0; i < n; ++i) {
    BatchPlan& p = B->plans[i];
    ferrox_ctx& c = p.c;
    auto c64 = level_coefficients<double>(&c);
    for (int k = 0; k < c.nz; ++k) coef0.push_back(c64[k]);
    const int dl = dense_level(&c);
    inst[i].dense_lev = dl;
    inst[i].dense_off = (long long)(denseT.size() / tsz);
    if (B->mixed) {
      auto c32 = level_coefficients<float>(&c);
      const unsigned char* q = reinterpret_cast<const unsigned char*>(c32.data());
      coefT.insert(coefT.end(), q, q + c32.size() * sizeof(PlaneCoef<float>));
      if (dl >= 0) {
        const auto inv = dense_inverse<float>(c32, c.lv_tail[dl]);
        const unsigned char* d = reinterpret_cast<const unsigned char*>(inv.data());
        denseT.insert(denseT.end(), d, d + inv.size() * sizeof(float));
      }
    } else {
      const unsigned char* q = reinterpret_cast<const unsigned char*>(c64.data());
      coefT.insert(coefT.end(), q, q + c64.size() * sizeof(PlaneCoef<double>));
      if (dl >= 0) {
        const auto inv = dense_inverse<double>(c64, c.lv_tail[dl]);
        const unsigned char* d = reinterpret_cast<const unsigned char*>(inv.data());
        denseT.insert(denseT.end(), d, d + inv.size() * sizeof(double));
      }
    }
    planes.insert(planes.end(), c.planes.begin(), c.planes.end());
    for (auto L : c.lv) { L.off += p.arena_off; L.coef_off += p.coef_off; lv.push_back(L); }
    for (auto L : c.lv_tail) { L.coef_off += p.coef_off; lvt.push_back(L); }
    BatchInst& I = inst[i];
    I.P = B->P + p.cell_off;
    I.Pbuf = B->Pbuf + p.cell_off;
    I.phi = B->phi + p.cell_off;
    I.clamp = update_clamp(&c);
    I.fe_lo = c.fe_lo; I.fe_hi = c.fe_hi;
    I.lv_off = p.lv_off; I.nlev = (int)c.lv.size(); I.tail_first = c.tail_first;
    I.lvt_off = p.lvt_off; I.nlev_tail = (int)c.lv_tail.size();
    I.bottom_sweeps = c.num.bottom_sweeps;
    I.tail_elems = c.tail_elems;
    I.tail_base = c.lv[c.tail_first].off + p.arena_off;
    TDGLArgs& t = I.tdgl;
    t.P_in = I.P; t.P_out = I.Pbuf; t.P_base = nullptr; t.F_store = nullptr;
    t.phi = I.phi; t.b = B->b + p.cell_off; t.planes = B->planes + p.plane_off; t.params = B->params + i;
    t.nx = c.nx; t.ny = c.ny; t.nz = c.nz; t.ncomp = 1; t.kd_lo = c.kd_lo; t.kd_hi = c.kd_hi;
    t.dt = num->dt; t.inv_h = 1.0 / c.h; t.inv_h2 = 1.0 / (c.h * c.h); t.b_scale = c.h / kEps0; t.mode = 0;
    ResidArgs& ra = I.resid;
    ra.phi = I.phi; ra.b = t.b; ra.planes = t.planes; ra.coef0 = B->coef0 + p.coef0_off; ra.params = t.params;
    ra.nx = c.nx; ra.ny = c.ny; ra.nz = c.nz;
    ra.r_out = static_cast<char*>(B->r) + (size_t)p.arena_off * tsz;
    ra.s_out = has_sc && c.has_sc ? static_cast<char*>(B->s) + (size_t)p.arena_off * tsz : nullptr;
    ra.carriers = carrier_kind(&c);
    // FP64 residual: measured, the double-float form is slower in the batched
    // residual, whose columns give too few threads to hide its longer chains (64
    // instances: 1004 against 1091 Mcell-steps/s in the persistent launch, 1048
    // against 1111 in the graph of phases)
    ra.coef_df = nullptr;
    ra.partials = nullptr;
    ra.stats = B->stats + i;
    ra.tol = num->tol; ra.max_cycles = num->max_cycles; ra.first = 1; ra.set_cond = 0;
    ra.cond_handle = 0; ra.launches_per_cycle = 0; ra.kchunk = c.nz;
  }
  FX_BINIT(cudaMemcpy(B->coef, coefT.data(), coefT.size(), cudaMemcpyHostToDevice));
  if (!denseT.empty()) {
    FX_BINIT(cudaMalloc(&B->dense, denseT.size()));
    FX_BINIT(cudaMemcpy(B->dense, denseT.data(), denseT.size(), cudaMemcpyHostToDevice));
  }
  FX_BINIT(cudaMemcpy(B->coef0, coef0.data(), coef0.size() * sizeof(PlaneCoef<double>), cudaMemcpyHostToDevice));
  FX_BINIT(cudaMemcpy(B->planes, planes.data(), planes.size() * sizeof(PlaneTDGL), cudaMemcpyHostToDevice));
  FX_BINIT(cudaMemcpy(B->lv, lv.data(), lv.size() * sizeof(LevelDesc), cudaMemcpyHostToDevice));
  FX_BINIT(cudaMemcpy(B->lvt, lvt.data(), lvt.size() * sizeof(LevelDesc), cudaMemcpyHostToDevice));
  FX_BINIT(cudaMemcpy(B->inst, inst.data(), n * sizeof(BatchInst), cudaMemcpyHostToDevice));
  FX_BINIT(cudaMemset(B->b, 0, cells * sizeof(double)));
  FX_BINIT(cudaMemset(B->Pbuf, 0, cells * sizeof(double)));
  FX_BINIT(cudaMemset(B->e, 0, arena * tsz));
  FX_BINIT(cudaMemset(B->r, 0, arena * tsz));
  if (B->s) FX_BINIT(cudaMemset(B->s, 0, arena * tsz));
  FX_BINIT(cudaMemset(B->bar, 0, (size_t)n * sizeof(GridBar)));
  FX_BINIT(cudaMemset(B->status, 0, sizeof(int)));
  FX_BINIT(cudaMemset(B->stats, 0, n * sizeof(DevStats)));
  FX_BINIT(cudaMemset(B->params, 0, n * sizeof(DevParams)));
  FX_BINIT(B->mixed ? batch_prepare<float>(B->smem) : batch_prepare<double>(B->smem));
  FX_BINIT(B->mixed ? phase_prepare<float>(B->smem) : phase_prepare<double>(B->smem));
  ferrox_status rc = batch_configure(B, 512, 1);
  if (rc != FERROX_OK) return cleanup(rc);
  FX_BINIT(cudaDeviceSynchronize());
#undef FX_BINIT
  *out = B;
  return FERROX_OK;
}

ferrox_status ferrox_batch_set_bias(ferrox_batch* B, const double* v_bottom, const double* v_top) {
  if (!B || !v_bottom || !v_top) return bfail(B, FERROX_EINVAL, "null argument");
  std::vector<DevParams> p(B->n);
  for (int i = 0; i < B->n; ++i) {
    if (!std::isfinite(v_bottom[i]) || !std::isfinite(v_top[i])) return bfail(B, FERROX_EINVAL, "bias not finite");
    p[i].v_bot = v_bottom[i];
    p[i].v_top = v_top[i];
  }
  // pageable source: staged before the call returns
  FX_BCK(cudaMemcpyAsync(B->params, p.data(), B->n * sizeof(DevParams), cudaMemcpyHostToDevice, B->stream));
  return FERROX_OK;
}

ferrox_status ferrox_batch_solve_poisson(ferrox_batch* B) {
  if (!B) return bfail(nullptr, FERROX_EINVAL, "null batch");
  if (B->ge_solve) FX_BCK(cudaGraphLaunch(B->ge_solve, B->stream));
  else FX_BCK(batch_launch(B, 1, B->stream));
  return FERROX_OK;
}

ferrox_status ferrox_batch_step(ferrox_batch* B, int nsteps) {
  if (!B) return bfail(nullptr, FERROX_EINVAL, "null batch");
  if (nsteps < 0) return bfail(B, FERROX_EINVAL, "nsteps < 0");
  if (nsteps == 0) return FERROX_OK;
  if (!B->tuned) {
    ferrox_status rc = batch_autotune(B);
    if (rc != FERROX_OK) return rc;
    rc = batch_build_graphs(B);
    if (rc != FERROX_OK) return rc;
    B->tuned = true;
  }
  if (B->engine == 1) {   // the phase graph is one step
    for (int k = 0; k < nsteps; ++k) FX_BCK(cudaGraphLaunch(B->ge_step, B->stream));
    return FERROX_OK;
  }
  // pageable source: staged before the call returns, so the graph reads this count
  FX_BCK(cudaMemcpyAsync(B->nsteps_d, &nsteps, sizeof(int), cudaMemcpyHostToDevice, B->stream));
  FX_BCK(cudaGraphLaunch(B->ge_step, B->stream));
  return FERROX_OK;
}

ferrox_status ferrox_batch_stats(ferrox_batch* B, ferrox_stats* out) {
  if (!B || !out) return bfail(B, FERROX_EINVAL, "null argument");
  std::vector<DevStats> st(B->n);
  int gst = 0;
  FX_BCK(cudaMemcpyAsync(st.data(), B->stats, B->n * sizeof(DevStats), cudaMemcpyDeviceToHost, B->stream));
  FX_BCK(cudaMemcpyAsync(&gst, B->status, sizeof(int), cudaMemcpyDeviceToHost, B->stream));
  FX_BCK(cudaStreamSynchronize(B->stream));
  ferrox_status worst = (ferrox_status)gst;
  for (int i = 0; i < B->n; ++i) {
    out[i].steps = st[i].steps;
    out[i].launches = st[i].steps;
    out[i].solves = st[i].solves;
    out[i].cycles = st[i].cycles;
    out[i].vcycles = st[i].vcycles;
    out[i].nn_rejected = 0;
    out[i].last_cycles = st[i].last_cycles;
    out[i].last_rel_res = st[i].last_rel;
    out[i].status = gst ? gst : st[i].status;
    if (worst == FERROX_OK && st[i].status) worst = (ferrox_status)st[i].status;
  }
  if (worst != FERROX_OK) B->err = worst == FERROX_ETIMEOUT ? "a bounded grid barrier ran out of time"
                                                            : "an instance reported a device error";
  return worst;
}

ferrox_status ferrox_batch_charge(ferrox_batch* B, ferrox_charge_t* out) {
  if (!B || !out) return bfail(B, FERROX_EINVAL, "null argument");
  std::vector<DevParams> prm(B->n);
  FX_BCK(cudaMemcpyAsync(prm.data(), B->params, B->n * sizeof(DevParams), cudaMemcpyDeviceToHost, B->stream));
  for (int i = 0; i < B->n; ++i) {
    const ferrox_ctx& c = B->plans[i].c;
    ChargeArgs a{};
    a.phi = B->phi + B->plans[i].cell_off;
    a.P = B->P + B->plans[i].cell_off;
    a.planes = B->planes + B->plans[i].plane_off;
    a.params = B->params + i;
    a.nx = c.nx; a.ny = c.ny; a.nz = c.nz; a.k_int = c.k_int;
    a.h = c.h; a.eps0 = kEps0;
    a.eps_top = kEps0 * c.epsr[c.nz - 1];
    a.eps_bot = kEps0 * c.epsr[0];
    a.eps_L = c.k_int > 0 ? kEps0 * c.epsr[c.k_int - 1] : 0.0;
    a.eps_R = kEps0 * c.epsr[c.k_int];
    a.out = B->charge_out + 8 * i;
    a.partials = B->charge_part + (size_t)4 * 64 * i;
    launch_charge(a, B->stream);
  }
  FX_BCK(cudaGetLastError());
  FX_BCK(cudaMemcpyAsync(B->host_pinned, B->charge_out, (size_t)B->n * 8 * sizeof(double),
                         cudaMemcpyDeviceToHost, B->stream));
  FX_BCK(cudaStreamSynchronize(B->stream));
  for (int i = 0; i < B->n; ++i) {
    const ferrox_ctx& c = B->plans[i].c;
    const double* s = B->host_pinned + 8 * i;
    const double inv = 1.0 / ((double)c.nx * c.ny);
    out[i].Q_int = -s[0] * inv;
    out[i].phi_int_avg = s[1] * inv;
    out[i].V_fe = prm[i].v_top - out[i].phi_int_avg;
    out[i].sigma_top = -s[2] * inv;
    out[i].sigma_bot = s[3] * inv;
  }
  std::vector<ferrox_stats> st(B->n);
  return ferrox_batch_stats(B, st.data());
}

ferrox_status ferrox_batch_tuning(const ferrox_batch* B, int* threads, int* rows_per_unit, int* blocks) {
  if (!B) return FERROX_EINVAL;
  if (threads) *threads = B->threads;
  if (rows_per_unit) *rows_per_unit = B->rows_per_unit;
  if (blocks) *blocks = B->engine == 1 ? B->unit_blocks : B->blocks;
  return B->tuned ? FERROX_OK : FERROX_ESTATE;
}

ferrox_status ferrox_batch_engine(const ferrox_batch* B, int* engine) {
  if (!B || !engine) return FERROX_EINVAL;
  *engine = B->engine;
  return B->tuned ? FERROX_OK : FERROX_ESTATE;
}

ferrox_status ferrox_batch_set_engine(ferrox_batch* B, int engine) {
  if (!B) return bfail(nullptr, FERROX_EINVAL, "null batch");
  if (engine != 0 && engine != 1) return bfail(B, FERROX_EINVAL, "engine must be 0 or 1");
  FX_BCK(cudaStreamSynchronize(B->stream));
  B->engine = engine;
  const ferrox_status rc0 = engine == 1 ? phase_configure(B)
                                        : batch_configure(B, B->threads, B->rows_per_unit, 1, B->grouped);
  if (rc0 != FERROX_OK) return rc0;
  if (B->ge_step) { cudaGraphExecDestroy(B->ge_step); B->ge_step = nullptr; }
  if (B->ge_solve) { cudaGraphExecDestroy(B->ge_solve); B->ge_solve = nullptr; }
  if (B->gr_step) { cudaGraphDestroy(B->gr_step); B->gr_step = nullptr; }
  if (B->gr_solve) { cudaGraphDestroy(B->gr_solve); B->gr_solve = nullptr; }
  const ferrox_status rc = batch_build_graphs(B);
  if (rc != FERROX_OK) return rc;
  B->tuned = true;
  return FERROX_OK;
}

ferrox_status ferrox_batch_set_shape(ferrox_batch* B, int threads, int rows_per_unit,
                                     int ctas_per_sm, int grouped) {
  if (!B) return bfail(nullptr, FERROX_EINVAL, "null batch");
  if ((threads != 256 && threads != 512) ||
      (rows_per_unit != 1 && rows_per_unit != 2 && rows_per_unit != 4) || ctas_per_sm < 1 ||
      (grouped != 0 && grouped != 1))
    return bfail(B, FERROX_EINVAL, "bad launch shape");
  int per_sm = 0;
  FX_BCK(B->mixed ? batch_occupancy<float>(threads, B->smem, &per_sm)
                  : batch_occupancy<double>(threads, B->smem, &per_sm));
  if (ctas_per_sm > per_sm) return bfail(B, FERROX_EINVAL, "that many CTAs per SM do not fit");
  FX_BCK(cudaStreamSynchronize(B->stream));
  B->engine = 0;
  ferrox_status rc = batch_configure(B, threads, rows_per_unit, ctas_per_sm, grouped);
  if (rc != FERROX_OK) return rc;
  if (B->ge_step) { cudaGraphExecDestroy(B->ge_step); B->ge_step = nullptr; }
  if (B->ge_solve) { cudaGraphExecDestroy(B->ge_solve); B->ge_solve = nullptr; }
  if (B->gr_step) { cudaGraphDestroy(B->gr_step); B->gr_step = nullptr; }
  if (B->gr_solve) { cudaGraphDestroy(B->gr_solve); B->gr_solve = nullptr; }
  rc = batch_build_graphs(B);
  if (rc != FERROX_OK) return rc;
  B->tuned = true;
  return FERROX_OK;
}

static_assert(kPhaseClasses == FERROX_PHASE_CLASSES, "phase classes of the header and the engine");

ferrox_status ferrox_batch_profile_phases(ferrox_batch* B, double* ms_out, int* launches_out) {
  if (!B || !ms_out || !launches_out) return bfail(B, FERROX_EINVAL, "null argument");
  if (!B->tuned || B->engine != 1)
    return bfail(B, FERROX_ESTATE,
                 "the phase profile runs the graph engine's kernels: tune it first or set engine 1");
  for (int q = 0; q < kPhaseClasses; ++q) {
    ms_out[q] = 0.0;
    launches_out[q] = 0;
  }
  FX_BCK(cudaStreamSynchronize(B->stream));
  const BatchArgs a = batch_args(B, 0);
  FX_BCK(B->mixed ? profile_phases<float>(a, B->unit_blocks, B->smem, B->stream, B->any_d, B->any_h,
                                          B->num.max_cycles, ms_out, launches_out)
                  : profile_phases<double>(a, B->unit_blocks, B->smem, B->stream, B->any_d, B->any_h,
                                           B->num.max_cycles, ms_out, launches_out));
  return FERROX_OK;
}

ferrox_status ferrox_batch_groups(const ferrox_batch* B, int* ngroups) {
  if (!B || !ngroups) return FERROX_EINVAL;
  *ngroups = B->ngroups;
  return B->tuned ? FERROX_OK : FERROX_ESTATE;
}

ferrox_status ferrox_check_wait_timeout(double seconds, int* status_out, void* cuda_stream) {
  ferrox_batch* B = nullptr;
  if (!status_out || !(seconds > 0.0) || seconds > 5.0) return bfail(nullptr, FERROX_EINVAL, "bad argument");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  GridBar* gb = nullptr;
  int* st = nullptr;
  FX_BCK(cudaMalloc(&gb, sizeof(GridBar)));
  FX_BCK(cudaMalloc(&st, sizeof(int)));
  FX_BCK(cudaMemsetAsync(gb, 0, sizeof(GridBar), s));
  FX_BCK(cudaMemsetAsync(st, 0, sizeof(int), s));
  FX_BCK(launch_barrier_timeout(gb, st, (long long)(seconds * 2.0e9), s));
  FX_BCK(cudaMemcpyAsync(status_out, st, sizeof(int), cudaMemcpyDeviceToHost, s));
  FX_BCK(cudaStreamSynchronize(s));
  cudaFree(gb);
  cudaFree(st);
  return FERROX_OK;
}

ferrox_status ferrox_carrier_exp(const double* u_dev, double* ep_dev, double* em_dev, long long n,
                                 void* cuda_stream) {
  ferrox_batch* B = nullptr;
  if (n < 0 || (n > 0 && (!u_dev || !ep_dev || !em_dev))) return bfail(nullptr, FERROX_EINVAL, "bad argument");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  FX_BCK(launch_carrier_exp(u_dev, ep_dev, em_dev, n, s));
  FX_BCK(cudaStreamSynchronize(s));
  return FERROX_OK;
}

ferrox_status ferrox_carrier_exp_df(const float* u_hl_dev, double* ep_dev, double* em_dev, long long n,
                                    void* cuda_stream) {
  ferrox_batch* B = nullptr;
  if (n < 0 || (n > 0 && (!u_hl_dev || !ep_dev || !em_dev))) return bfail(nullptr, FERROX_EINVAL, "bad argument");
  if (reinterpret_cast<uintptr_t>(u_hl_dev) % 8) return bfail(nullptr, FERROX_EINVAL, "u_hl must be 8-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  FX_BCK(launch_carrier_exp_df(u_hl_dev, ep_dev, em_dev, n, s));
  FX_BCK(cudaStreamSynchronize(s));
  return FERROX_OK;
}

// self-check record of the last persistent launch: [0] set when a wait ran out,
// [1] its barrier number, [2] the waiting block, [3] arrivals seen, [4] generation,
// [8 + b] barriers block b passed (negative: it left on a failed wait)
ferrox_status ferrox_batch_debug(ferrox_batch* B, int* out, int n) {
  if (!B || !out || n < 8) return FERROX_EINVAL;
  FX_BCK(cudaMemcpy(out, B->dbg, std::min(n, 8 + 1024) * sizeof(int), cudaMemcpyDeviceToHost));
  return FERROX_OK;
}

ferrox_status ferrox_batch_destroy(ferrox_batch* B) {
  batch_release(B);
  return FERROX_OK;
}

const char* ferrox_batch_last_error(const ferrox_batch* B) {
  return B ? B->err.c_str() : g_init_error.c_str();
}

}  // extern "C"

// ---- entry point without allocation -----------------------------------------------------
//
// Callers that cannot allocate device memory (processes held to a fixed
// device-memory budget, frameworks whose own allocator must own every device
// byte, or latency-bound loops that cannot afford the device-wide
// synchronisation cudaMalloc and cudaFree may imply) still need the TDGL
// update.  ferrox_tdgl_update_static runs the same fused TDGL kernel as
// ferrox_tdgl_update, with its three scratch areas (plane table, staging copy
// of the new polarization, right-hand side) carved from the file-scope array
// below, which every GPU that loads the library holds until the process exits.
namespace {

constexpr long long kStaticMaxCells = FERROX_STATIC_MAX_CELLS;
constexpr int kStaticMaxPlanes = FERROX_STATIC_MAX_PLANES;
constexpr size_t kStaticPlaneBytes = ((size_t)kStaticMaxPlanes * sizeof(PlaneTDGL) + 255) / 256 * 256;
constexpr size_t kStaticParamBytes = 256;
constexpr size_t kStaticStateBytes = (size_t)kStaticMaxCells * 4 * sizeof(double);  // 3 comps + b
constexpr size_t kStaticBytes = kStaticParamBytes + kStaticPlaneBytes + kStaticStateBytes;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

std::mutex g_static_mu;
unsigned char* g_static_ptr[64] = {};   // device address of g_static_scratch, per device

// Plane table of the static path, written into a caller-side array without any
// heap use; the same per-plane quantities as the context path.
ferrox_status static_planes(const ferrox_geometry* g, PlaneTDGL* out, int* nz_out, int* fe_lo,
                            int* fe_hi) {
  int nz = 0;
  for (int q = 0; q < g->nlayers; ++q) nz += g->layers[q].ncells;
  if (nz > kStaticMaxPlanes) return FERROX_EINVAL;
  const double h = g->h;
  double kappa;
  if (g->pbc == FERROX_PBC_FREE) kappa = 1.0 / 8.0;
  else if (g->pbc == FERROX_PBC_ZERO) kappa = 0.0;
  else kappa = g->lambda / (3.0 * h + 8.0 * g->lambda);
  int z = 0;
  *fe_lo = nz;
  *fe_hi = -1;
  for (int q = 0; q < g->nlayers; ++q) {
    const ferrox_layer& L = g->layers[q];
    for (int c = 0; c < L.ncells; ++c, ++z) {
      PlaneTDGL p{};
      p.eps_r = L.eps_r;
      p.fe = L.kind == FERROX_FE;
      if (p.fe) {
        p.alpha = L.alpha; p.beta = L.beta; p.gamma = L.gamma;
        p.alpha_xy = L.alpha_xy; p.beta_xy = L.beta_xy; p.gamma_xy = L.gamma_xy;
        p.g11 = L.g11; p.g44 = L.g44; p.Gamma = L.Gamma;
        *fe_lo = std::min(*fe_lo, z);
        *fe_hi = std::max(*fe_hi, z);
      }
      out[z] = p;
    }
  }
  for (z = 0; z < nz; ++z) {
    PlaneTDGL& p = out[z];
    const bool dn = z > 0 && out[z - 1].fe, up = z < nz - 1 && out[z + 1].fe;
    p.b_dyn = p.fe || dn || up;
    if (p.fe) {
      const double ih2 = 1.0 / (h * h);
      if (dn && up) {
        p.wz_dn = ih2; p.wz_c = -2.0 * ih2; p.wz_up = ih2;
      } else if (up || dn) {
        const double wn = 4.0 * (1.0 - 2.0 * kappa) / 3.0 * ih2;
        p.wz_c = 4.0 * (18.0 * kappa - 3.0) / 3.0 * ih2;
        p.wz_up = up ? wn : 0.0;
        p.wz_dn = dn ? wn : 0.0;
      } else {
        return FERROX_EINVAL;
      }
    }
    if (z > 0) {
      const double eL = out[z - 1].eps_r, eR = p.eps_r;
      p.fw_L = eL / (eL + eR);
      p.fw_R = eR / (eL + eR);
      p.fpc = h / (2.0 * kEps0 * (eL + eR));
    }
    p.lift = (z == 0 || z == nz - 1) ? 2.0 * p.eps_r : 0.0;
  }
  *nz_out = nz;
  return FERROX_OK;
}

}  // namespace

extern "C" ferrox_status ferrox_tdgl_update_static(const ferrox_geometry* geom, double dt,
                                                   double v_bottom, double v_top, double* P_dev,
                                                   const double* phi_dev, void* cuda_stream) {
  auto bad = [](const char* m) { return fail(nullptr, FERROX_EINVAL, m); };
  if (!geom || !geom->layers || geom->nlayers < 1 || !P_dev || !phi_dev) return bad("null argument");
  if ((reinterpret_cast<uintptr_t>(P_dev) | reinterpret_cast<uintptr_t>(phi_dev)) % 8)
    return bad("state arrays must be 8-byte aligned");
  if (geom->nx < 1 || geom->ny < 1 || !(geom->h > 0.0) || !(dt > 0.0)) return bad("bad sizes");
  if ((geom->nx != 1 && geom->nx % 2) || (geom->ny != 1 && geom->ny % 2))
    return bad("lateral sizes must be even or 1");
  if (geom->ncomp != 1 && geom->ncomp != 3) return bad("ncomp must be 1 or 3");
  if (!std::isfinite(v_bottom) || !std::isfinite(v_top)) return bad("bias not finite");
  long long nzl = 0;
  for (int q = 0; q < geom->nlayers; ++q) {
    if (geom->layers[q].ncells < 1 || !(geom->layers[q].eps_r > 0.0)) return bad("bad layer");
    nzl += geom->layers[q].ncells;
  }
  const long long N = (long long)geom->nx * geom->ny * nzl;
  if (N > kStaticMaxCells || nzl > kStaticMaxPlanes)
    return bad("ferrox_tdgl_update_static: grid larger than its static scratch "
               "(at most FERROX_STATIC_MAX_CELLS cells and FERROX_STATIC_MAX_PLANES planes)");
  PlaneTDGL planes[kStaticMaxPlanes];
  int nz = 0, fe_lo = 0, fe_hi = -1;
  if (static_planes(geom, planes, &nz, &fe_lo, &fe_hi) != FERROX_OK || fe_hi < 0)
    return bad("the stack needs a ferroelectric layer at least 2 cells thick");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) return fail(nullptr, FERROX_ECUDA, "cudaGetDevice failed");
  unsigned char* base;
  {
    // set-up once per device, with that device current: the host-side name of
    // the array is not a device address, so ask the runtime for it
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_static_scratch);
      if (e != cudaSuccess)
        return fail(nullptr, FERROX_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_static_ptr[dev] = static_cast<unsigned char*>(ptr);
    }
    base = g_static_ptr[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  DevParams* params = reinterpret_cast<DevParams*>(base);
  PlaneTDGL* planes_d = reinterpret_cast<PlaneTDGL*>(base + kStaticParamBytes);
  double* Pout = reinterpret_cast<double*>(base + kStaticParamBytes + kStaticPlaneBytes);
  double* b = Pout + (size_t)geom->ncomp * N;
  // pageable source: the copy is staged before the call returns
  e = cudaMemcpyAsync(planes_d, planes, nz * sizeof(PlaneTDGL), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return fail(nullptr, FERROX_ECUDA, std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e));
  launch_set_params(params, v_bottom, v_top, s);
  TDGLArgs a{};
  a.P_in = P_dev; a.P_out = Pout; a.P_base = nullptr; a.F_store = nullptr;
  a.phi = phi_dev; a.b = b; a.planes = planes_d; a.params = params;
  a.nx = geom->nx; a.ny = geom->ny; a.nz = nz; a.ncomp = geom->ncomp;
  a.kd_lo = std::max(0, fe_lo - 1);
  a.kd_hi = std::min(nz - 1, fe_hi + 1);
  a.dt = dt; a.inv_h = 1.0 / geom->h; a.inv_h2 = 1.0 / (geom->h * geom->h);
  a.b_scale = geom->h / kEps0;
  a.mode = 0;
  launch_tdgl(a, s);
  // The kernel writes the new polarization on ferroelectric planes only, so copy
  // back each contiguous run of them on its own: the staging area keeps whatever
  // an earlier call left on the other planes, and the caller's planes between two
  // ferroelectric layers must not receive it.
  const long long plane = (long long)geom->nx * geom->ny;
  for (int z0 = fe_lo; z0 <= fe_hi;) {
    if (!planes[z0].fe) { ++z0; continue; }
    int z1 = z0;
    while (z1 + 1 <= fe_hi && planes[z1 + 1].fe) ++z1;
    const size_t off = (size_t)z0 * plane, cnt = (size_t)(z1 - z0 + 1) * plane;
    for (int q = 0; q < geom->ncomp; ++q) {
      e = cudaMemcpyAsync(P_dev + q * N + off, Pout + q * N + off, cnt * sizeof(double),
                          cudaMemcpyDeviceToDevice, s);
      if (e != cudaSuccess)
        return fail(nullptr, FERROX_ECUDA, std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e));
    }
    z0 = z1 + 1;
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(nullptr, FERROX_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
  return FERROX_OK;
}

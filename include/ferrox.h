/*
 * ferrox.h -- C ABI of the GB300 (sm_103a) TDGL + Poisson time-step library.
 *
 * The library advances the self-consistent ferroelectric device model of
 * FerroX (arXiv 2210.15668): the time-dependent Ginzburg-Landau equation for
 * the polarization (Eq. TDGL2) coupled to the variable-permittivity Poisson
 * equation div(eps grad Phi) = div P - rho (Eq. Poisson), with the carrier
 * charge of semiconductor layers (Eq. rho; Boltzmann, Eq. MaxBolt_ne_np, or
 * Fermi-Dirac, Eqs. ne and np), periodic x/y
 * boundaries and Dirichlet electrodes (Methods, "Electrical boundary
 * conditions").  One context holds one device stack on one GPU.
 *
 * Conventions for every entry point:
 *   - Units are SI: metres, volts, C/m^2, F/m (eps = eps_r * eps0), seconds.
 *   - Arrays are C-contiguous float64 with x fastest:
 *       P   : [ncomp][Nz][Ny][Nx]  (ncomp = 1: P_z only; ncomp = 3: P_x, P_y, P_z)
 *       phi : [Nz][Ny][Nx]
 *     Nz is the sum of the layers' ncells; layers are listed bottom to top.
 *   - Pointers named *_dev are device pointers owned by the caller; they are
 *     registered at init and must stay valid until ferrox_destroy.  Pointers
 *     named *_host are host pointers (pinned memory gives asynchronous copies).
 *   - All work is enqueued on the CUDA stream given at init (NULL = legacy
 *     default stream) and returns without waiting, unless stated otherwise.
 *   - Every call returns a ferrox_status and never aborts.  Argument errors
 *     are reported at once.  Device-side conditions (multigrid or Newton not
 *     converged, a non-finite residual, a device wait that ran out of time)
 *     are recorded in a sticky device status word and reported by the next
 *     synchronising call (ferrox_sync_stats, ferrox_charge, ferrox_get_state).
 *     ferrox_last_error() describes the last failure in words.
 *   - Scratch memory (the multigrid hierarchy, right-hand side, CUDA graphs) is
 *     allocated by the library at init and freed by ferrox_destroy.
 *   - A context is not thread-safe: one host thread at a time per context.
 */
#ifndef FERROX_H
#define FERROX_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ferrox_ctx ferrox_ctx; /* opaque */

typedef enum {
  FERROX_OK = 0,
  FERROX_EINVAL = 1,     /* invalid argument (reported synchronously) */
  FERROX_ENOMEM = 2,     /* device or host allocation failed */
  FERROX_ECUDA = 3,      /* a CUDA runtime call failed */
  FERROX_ENOCONV = 4,    /* multigrid / Newton reached max_cycles above tolerance */
  FERROX_ENONFINITE = 5, /* NaN or Inf in a residual norm */
  FERROX_ETIMEOUT = 6,   /* a bounded device wait ran out (batched persistent kernel) */
  FERROX_ESTATE = 7      /* call not valid in the context's current state */
} ferrox_status;

/* Material kinds of a layer (Fig. 1a: ferroelectric, dielectric, semiconductor). */
enum { FERROX_FE = 0, FERROX_DE = 1, FERROX_SC = 2 };

/* Polarization boundary condition at ferroelectric faces (Methods, Eqs. Pbc,
 * PbcFree, PbcDir): lambda dP/dn_in = P, its lambda -> infinity limit dP/dn = 0,
 * and its lambda = 0 limit P = 0.  Each is imposed through a second-order
 * one-sided three-point stencil. */
enum { FERROX_PBC_FREE = 0, FERROX_PBC_ZERO = 1, FERROX_PBC_LAMBDA = 2 };

/* Arithmetic of the Poisson solve: FP64 multigrid, or FP32 multigrid cycles
 * inside an FP64 defect-correction loop (FP64 residual, potential, norms and
 * carrier exponentials).  All stop on the same FP64 residual test.
 *   FERROX_FP64: V-cycles on phi itself, the residual norm fused into the
 *     fine-level restriction after the pre-smoothing (the test accepts phi after
 *     that pre-smoothing), when the stack has no semiconductor layer, inner is
 *     0 or 1 and the fine level coarsens in x, y and z; otherwise as
 *     FERROX_FP64_DEFECT.
 *   FERROX_FP64_DEFECT: FP64 V-cycles on the correction equation inside the
 *     defect-correction (Newton) loop, the residual computed by its own kernel
 *     before every V-cycle.
 * The batched engine runs the defect-correction form for FERROX_FP64. */
enum { FERROX_FP64 = 0, FERROX_MIXED = 1, FERROX_FP64_DEFECT = 2 };

/* Carrier statistics of a semiconductor layer.
 *   FERROX_BOLTZMANN: the Maxwell-Boltzmann limit (Eq. MaxBolt_ne_np) with the
 *     intrinsic density n_i: n = n0 e^{Phi/V_T}, p = p0 e^{-Phi/V_T}, n0 p0 = n_i^2.
 *   FERROX_FERMI_DIRAC: the paper's Fermi-Dirac model (Eqs. ne, np), n = N_c
 *     F_1/2(eta_e), p = N_v F_1/2(eta_p), with N_c, N_v = 2 (2 pi m* k_B T/h^2)^{3/2}
 *     from the effective masses m_e, m_p and F_1/2 by the Bednarczyk approximation
 *     the paper uses (Methods, "Numerical Approach"); the band edges, E_g apart, are
 *     placed so that the bulk is neutral at Phi = 0.
 * Either way the bulk is neutral at Phi = 0 (ohmic contact at V0 = 0). */
enum { FERROX_BOLTZMANN = 0, FERROX_FERMI_DIRAC = 1 };

/* One planar layer (Table 1 lists the parameters).  Only the fields of its
 * kind are read: Landau/gradient/kinetic data for FE, carrier data for SC. */
typedef struct {
  int kind;                           /* FERROX_FE / _DE / _SC */
  int ncells;                         /* thickness in cells (>= 1; FE >= 2) */
  double eps_r;                       /* relative permittivity (> 0) */
  double alpha, beta, gamma;          /* Landau coefficients of P_z (Eq. free), SI */
  double alpha_xy, beta_xy, gamma_xy; /* Landau coefficients of P_x, P_y (ncomp = 3 only) */
  double g11, g44;                    /* gradient coefficients (Eq. grad): z, and x/y */
  double Gamma;                       /* kinetic coefficient (Eq. TDGL1) */
  double N_A, N_D;                    /* acceptor / donor density, m^-3 (SC) */
  double n_i;                         /* intrinsic carrier density, m^-3 (SC, Boltzmann) */
  double T;                           /* temperature, K (SC) */
  int stats;                          /* SC carrier statistics: FERROX_BOLTZMANN or
                                         FERROX_FERMI_DIRAC */
  int pad;
  double m_e, m_p;                    /* effective masses / m_e (SC, Fermi-Dirac; Table 1) */
  double E_g;                         /* band gap, eV (SC, Fermi-Dirac) */
} ferrox_layer;

typedef struct {
  int nx, ny;                  /* lateral cells; each even or 1 (periodic) */
  double h;                    /* cell size (uniform, m) */
  int nlayers;
  const ferrox_layer* layers;  /* bottom to top; copied at init */
  int pbc;                     /* FERROX_PBC_* */
  double lambda;               /* extrapolation length (m) for FERROX_PBC_LAMBDA */
  int ncomp;                   /* 1 (uniaxial, the paper's model) or 3 */
} ferrox_geometry;

typedef struct {
  double dt;        /* time step (s) */
  int order;        /* 1: predictor only (Steps 1a/1b); 2: with corrector (Steps 2a/2b) */
  double tol;       /* stop when ||r||_2 <= tol * max(||b||_2, ||rho||_2); e.g. 1e-10 */
  int nu1, nu2;     /* pre/post red-black Gauss-Seidel sweeps per V-cycle level */
  int max_cycles;   /* V-cycles (outer iterations) allowed per solve */
  int precision;    /* FERROX_FP64, FERROX_MIXED or FERROX_FP64_DEFECT */
  int bottom_sweeps;/* sweeps on the coarsest level (0: default) */
  int guess;        /* initial potential of each step's solve: 0 = the previous step's
                       potential (Step 1b of the Methods), 1 = linear extrapolation in
                       time 2 Phi^n - Phi^{n-1}.  The solve stops on the same residual
                       test either way; only the number of V-cycles changes. */
  int inner;        /* V-cycles per outer (defect-correction / Newton) iteration; 0 or 1:
                       one, the plain method.  The first starts from a zero correction,
                       the others continue it on the same right-hand side and Newton
                       shift, and phi is corrected once after the last: fewer FP64
                       residuals (and carrier exponentials) per solve.  inner < 0:
                       adaptive, at most -inner V-cycles, the count chosen on the device
                       after each residual from the contraction per V-cycle measured
                       over the previous outer iteration (kept across solves) and the
                       distance to the tolerance.  The stopping test is unchanged.
                       The batched engine takes 0 or 1 only. */
  int nonlinear;    /* iteration for the carrier charge rho(Phi) of semiconductor layers:
                       FERROX_NEWTON (damped Newton: the Jacobian's diagonal shift
                       q^2 (n + p)/kT in the multigrid operator) or FERROX_FIXED_POINT
                       (the paper's lagged fixed point, Methods "Numerical Approach":
                       each outer iteration relaxes A Phi = b + rho(Phi_k) with rho
                       frozen at the current Phi, no shift).  Both stop on the same
                       residual test and reach the same solution where they converge;
                       the fixed point converges only while the carrier response is
                       weak (undoped Si) and reports FERROX_ENOCONV otherwise.  The
                       batched engine takes FERROX_NEWTON only. */
  int tdgl_arith;   /* arithmetic of the TDGL force (Eq. TDGL2): FERROX_TDGL_FP64 (the
                       default) or FERROX_TDGL_FP32, which evaluates the force in FP32
                       from double-float splits of the FP64 state (every difference of
                       state values is formed before rounding to FP32) and advances the
                       FP64 polarization and right-hand side in FP64.  FP32 needs
                       precision FERROX_MIXED and one polarization component; the
                       batched engine takes FERROX_TDGL_FP64 only.  Accuracy: the
                       increment dt f agrees with FP64 to ~2e-7 of the largest
                       increment; over 100 steps of a run near P = 0 (where the
                       dynamics amplify differences) P agreed to 6.5e-7 and the
                       electrode charge to 1.2e-8 relative. */
} ferrox_numerics;

enum { FERROX_NEWTON = 0, FERROX_FIXED_POINT = 1 };
enum { FERROX_TDGL_FP64 = 0, FERROX_TDGL_FP32 = 1 };

typedef struct {
  double Q_int;        /* -<D_z> on the bottom face of the lowest FE plane (C/m^2) */
  double phi_int_avg;  /* mean potential on that face (V) */
  double V_fe;         /* v_top - phi_int_avg (V) */
  double sigma_top;    /* charge on the top electrode, -<D_z(top)> (C/m^2) */
  double sigma_bot;    /* charge on the bottom electrode, +<D_z(bottom)> (C/m^2) */
} ferrox_charge_t;

typedef struct {
  long long steps;         /* time steps taken */
  long long launches;      /* library kernels launched by steps and solves (device count) */
  long long solves;        /* Poisson solves run */
  long long cycles;        /* V-cycles (outer iterations) run, all solves */
  int last_cycles;         /* V-cycles of the most recent solve */
  double last_rel_res;     /* ||r|| / max(||b||, ||rho||) at the end of that solve */
  int status;              /* sticky device status (ferrox_status) */
  long long vcycles;       /* V-cycles run, all solves, inner cycles included (= cycles when
                              numerics.inner is 0 or 1) */
  long long nn_rejected;   /* learned corrections rejected because they did not lower ||r|| */
} ferrox_stats;

/* Create a context (a1: per-plane material tables, multigrid hierarchy, CUDA
 * graphs).  P_dev and phi_dev are the caller's state arrays (layout above);
 * their contents are not read until the first call that needs them.
 * Errors: EINVAL for a malformed geometry (Nz < 2, no FE layer, an FE layer
 * thinner than 2 cells, odd lateral size other than 1, h <= 0, eps_r <= 0,
 * ncomp not 1 or 3, misaligned pointers), ENOMEM, ECUDA. */
ferrox_status ferrox_init_geometry(ferrox_ctx** out, const ferrox_geometry* geom,
                                   const ferrox_numerics* num, double* P_dev,
                                   double* phi_dev, void* cuda_stream);

/* Electrode potentials Phi(z_min) = v_bottom, Phi(z_max) = v_top; V_app = v_top -
 * v_bottom (Methods, "Electrical boundary conditions").  Asynchronous. */
ferrox_status ferrox_set_bias(ferrox_ctx* ctx, double v_bottom, double v_top);

/* Step 0 of the Methods: solve the Poisson problem for the current P, starting
 * from the current phi (the paper starts from phi = 0), to the tolerance.
 * With semiconductor layers the carrier charge makes the problem nonlinear; it
 * is solved by damped Newton, each update from one multigrid cycle on the
 * Jacobian (diagonal shift q^2 (n + p)/kT in semiconductor cells). */
ferrox_status ferrox_solve_poisson(ferrox_ctx* ctx);

/* Step 1a alone: P <- P + dt f(P, phi) (Eq. TDGL2) on ferroelectric cells, and
 * the Poisson right-hand side for the new P.  No solve. */
ferrox_status ferrox_tdgl_update(ferrox_ctx* ctx);

/* Advance nsteps time steps: Steps 1a/1b (order 1) or 1a/1b/2a/2b (order 2),
 * each solve converged on the device (no host synchronisation). */
ferrox_status ferrox_step(ferrox_ctx* ctx, int nsteps);

/* Interface and electrode charges of the current state (Results, MFIM: Q and
 * V_fe).  Synchronises the stream; returns the sticky device status. */
ferrox_status ferrox_charge(ferrox_ctx* ctx, ferrox_charge_t* out);

/* The residual r = b + rho(Phi) - A Phi of the Poisson problem (Eq. Poisson in
 * the finite-volume form, scaled by h^2/eps0) for the current state: b is formed
 * from the current P and bias, rho from the current Phi.  r_host is a host array
 * of Nz*Ny*Nx doubles.  arithmetic selects how the stencil is evaluated:
 * FERROX_RESID_FP64 (the FP64 forms' outer residual) or
 * FERROX_RESID_DOUBLE_FLOAT (the mixed form's outer residual: double-float pairs
 * on the FP32 pipe, about 48 significant bits; r = h + l).  A diagnostic: it
 * allocates a device buffer, synchronises, and leaves the state unchanged (b is
 * recomputed from P, as every step does). */
enum { FERROX_RESID_FP64 = 0, FERROX_RESID_DOUBLE_FLOAT = 1 };
ferrox_status ferrox_residual(ferrox_ctx* ctx, int arithmetic, double* r_host);

/* A Q-V sweep (Results, MFIM: the triangular-wave voltage protocol of the Q-V
 * and Q-V_fe characteristics): for each point q < npoints, set the electrodes to
 * v_bottom = 0, v_top = v_app[q] (host array), advance steps_per_point time steps
 * and record the charges of the resulting state in out[q] (host array of
 * npoints).  The state carries over from point to point (the hysteresis depends
 * on the path).  Equivalent to the calls ferrox_set_bias / ferrox_step /
 * ferrox_charge in that order.  Synchronises once per point; EINVAL for npoints
 * < 1, steps_per_point < 0 or null arrays; stops at the first point whose
 * status is not FERROX_OK and returns that status (out[q] of later points
 * untouched). */
ferrox_status ferrox_qv_sweep(ferrox_ctx* ctx, const double* v_app, int npoints, int steps_per_point,
                              ferrox_charge_t* out);

/* Counters and the sticky status.  Synchronises the stream. */
ferrox_status ferrox_sync_stats(ferrox_ctx* ctx, ferrox_stats* out);

/* Clear the sticky device status (after the caller has handled it). */
ferrox_status ferrox_clear_status(ferrox_ctx* ctx);

/* Copy the state between the registered device arrays and host arrays of the
 * same layout (checkpoint / restart, and the host-buffer path of the API).
 * ferrox_get_state synchronises; ferrox_set_state is asynchronous, so the host
 * arrays must stay unchanged until the stream reaches the copy. Either host
 * pointer may be NULL to skip that array. */
ferrox_status ferrox_get_state(ferrox_ctx* ctx, double* P_host, double* phi_host);
ferrox_status ferrox_set_state(ferrox_ctx* ctx, const double* P_host, const double* phi_host);

/* The same copies with P restricted to the ferroelectric film, the planes
 * fe_lo..fe_hi that ferrox_fe_planes reports: P_fe_host is
 * [ncomp][fe_hi - fe_lo + 1][ny][nx].  Outside the film P is zero in the model
 * (Methods, TDGL: the polarization belongs to the FE layer), so this is the whole
 * state at a third of the bytes for the 10-of-32-plane stacks; the device planes
 * outside the film keep their values (zero unless ferrox_set_state wrote others).
 * Synchronisation as for ferrox_get_state / ferrox_set_state. */
ferrox_status ferrox_fe_planes(const ferrox_ctx* ctx, int* fe_lo, int* fe_hi);
ferrox_status ferrox_get_state_fe(ferrox_ctx* ctx, double* P_fe_host, double* phi_host);
ferrox_status ferrox_set_state_fe(ferrox_ctx* ctx, const double* P_fe_host, const double* phi_host);

/* Kernel classes reported by ferrox_profile_step. */
enum {
  FERROX_K_TDGL = 0,      /* fused TDGL update + right-hand side */
  FERROX_K_RESID = 1,     /* FP64 outer residual, carrier charge, norms, convergence test */
  FERROX_K_SMOOTH0 = 2,   /* red-black Gauss-Seidel colour sweep on the fine level */
  FERROX_K_SMOOTHC = 3,   /* colour sweeps on coarser multi-block levels */
  FERROX_K_RESTRICT = 4,  /* residual + restriction */
  FERROX_K_PROLONG = 5,   /* prolongation + correction */
  FERROX_K_TAIL = 6,      /* single-CTA V-cycle over the smallest levels */
  FERROX_K_UPDATE = 7,    /* phi += correction */
  FERROX_K_COPY = 8,      /* copy of the new polarization; initial-guess extrapolation */
  FERROX_K_COUNT = 9
};

/* One time step run eagerly (no CUDA graph) with a CUDA event pair around every
 * launch, for a per-kernel time breakdown: on return ms[k] is the summed device
 * time and count[k] the number of launches of class k (arrays of FERROX_K_COUNT).
 * The launches between two host synchronisations (one V-cycle, or the TDGL
 * update) are queued behind a short untimed delay kernel, so the device runs
 * them back to back and the events time the kernels, not the host's launch
 * rate.  The result of the step is the same as ferrox_step(ctx, 1).
 * Synchronises. */
ferrox_status ferrox_profile_step(ferrox_ctx* ctx, double* ms, int* count);

/* The same step, also reporting in bytes[k] (array of FERROX_K_COUNT, may be
 * NULL) the algorithmic bytes of the class's launches: every array element the
 * method needs read or written once per launch (multigrid arrays in the
 * solve's precision, state and right-hand side in FP64; a dense bottom solve
 * counts its inverse once).  bytes[k] / ms[k] is the class's effective
 * bandwidth against the HBM roofline.  Synchronises. */
ferrox_status ferrox_profile_step_bytes(ferrox_ctx* ctx, double* ms, int* count, double* bytes);

/* Release everything the context allocated (the caller's arrays are untouched).
 * Synchronises the stream.  NULL is accepted. */
ferrox_status ferrox_destroy(ferrox_ctx* ctx);

/* Text of the last error of this context (or of the last failed init when ctx
 * is NULL).  The pointer stays valid until the next call on the context. */
const char* ferrox_last_error(const ferrox_ctx* ctx);

/* Multigrid hierarchy actually built: number of levels and, for level l < n,
 * its cell counts.  Returns EINVAL if l is out of range. */
ferrox_status ferrox_level_shape(const ferrox_ctx* ctx, int l, int* nx, int* ny, int* nz,
                                 int* nlevels);

/* ---- batched Q-V sweeps -----------------------------------------------------------------
 * n independent device stacks (instances) of possibly different lateral size,
 * stack and bias, advanced together: every phase of the time step runs over all
 * instances at once, and each instance checks its own convergence and drops out
 * when done.  Two engines (ferrox_batch_engine): ONE cooperative persistent
 * kernel per call with grid barriers between the phases, whose waits are
 * bounded in time (on expiry the launch records FERROX_ETIMEOUT instead of
 * hanging), or a CUDA graph of per-phase launches.  The engine and its shape
 * (threads per block, rows per work unit) are chosen by timing the candidates
 * on the first ferrox_batch_step, on a saved copy of the state that is
 * restored afterwards, and cached per problem shape.  This serves the Q-V
 * sweeps of the Results section (many biases and sizes). */
typedef struct ferrox_batch ferrox_batch; /* opaque */

/* Instances are uniaxial (ncomp = 1) and use order-1 steps.  P_dev and phi_dev
 * hold all instances back to back: instance i starts at element sum_{q<i} N_q,
 * N_q = Nx*Ny*Nz of instance q, with the per-instance layout above. */
ferrox_status ferrox_init_batch(ferrox_batch** out, int n, const ferrox_geometry* geoms,
                                const ferrox_numerics* num, double* P_dev, double* phi_dev,
                                void* cuda_stream);
/* Electrode potentials of every instance (arrays of n).  Asynchronous. */
ferrox_status ferrox_batch_set_bias(ferrox_batch* b, const double* v_bottom, const double* v_top);
/* Step 0 for every instance (one persistent launch, or the phase graph). */
ferrox_status ferrox_batch_solve_poisson(ferrox_batch* b);
/* nsteps time steps of every instance: one persistent launch, or nsteps launches
 * of the phase graph (see ferrox_batch_engine).  The first call autotunes. */
ferrox_status ferrox_batch_step(ferrox_batch* b, int nsteps);
/* Q, V_fe and electrode charges of every instance (array of n).  Synchronises. */
ferrox_status ferrox_batch_charge(ferrox_batch* b, ferrox_charge_t* out);
/* Counters and status of every instance (array of n).  Synchronises. */
ferrox_status ferrox_batch_stats(ferrox_batch* b, ferrox_stats* out);
/* The launch shape the autotuner chose (ESTATE before the first step); with the
 * phase graph, threads and blocks are those of its per-phase launches. */
ferrox_status ferrox_batch_tuning(const ferrox_batch* b, int* threads, int* rows_per_unit,
                                  int* blocks);
/* CTA groups of the tuned launch: 1 when every CTA works on every instance
 * behind one grid barrier; more when contiguous instance ranges run on their
 * own CTAs behind their own barriers. */
ferrox_status ferrox_batch_groups(const ferrox_batch* b, int* ngroups);
/* Fix the persistent engine and its launch shape instead of autotuning them:
 * threads per CTA (256 or 512), rows per work unit (1, 2 or 4), CTAs per SM
 * (1 .. what fits) and grouped (0: one grid barrier over every instance; 1: CTA
 * groups with their own barriers).  Every shape computes the same results; only
 * the speed differs. */
ferrox_status ferrox_batch_set_shape(ferrox_batch* b, int threads, int rows_per_unit,
                                     int ctas_per_sm, int grouped);
/* The engine the autotuner chose (ESTATE before the first step): 0 = one
 * persistent launch with grid barriers between its phases; 1 = a CUDA graph of
 * per-phase launches (TDGL, residual, per-instance decision, each level's colour
 * sweeps and transfers, the per-instance tails) whose solve loop is a WHILE node
 * the decision kernel sets while any instance is above the tolerance.  Both do
 * the same operations per cell in the same order and form the same per-instance
 * sums, so they give identical results; only the speed differs. */
ferrox_status ferrox_batch_engine(const ferrox_batch* b, int* engine);
/* Fix the engine instead of autotuning it (0 with the current shape at one CTA
 * per SM, or 1 with one row per work unit).  EINVAL for other values.
 * Synchronises. */
ferrox_status ferrox_batch_set_engine(ferrox_batch* b, int engine);
/* Classes of ferrox_batch_profile_phases, in this order: TDGL update, outer
 * residual, per-instance decisions, fine-level sweeps, coarser-level sweeps,
 * transfers (restriction and prolongation), tails, other (flags, counters). */
#define FERROX_PHASE_CLASSES 8
/* One time step of every instance with the graph engine's kernels launched one
 * by one (no graph), the solve loop driven from the host by the decision
 * kernel's "any instance active" flag: the same kernels in the same order as a
 * step of the graph, so the state advances exactly as ferrox_batch_step(b, 1)
 * would.  Each launch is timed by CUDA events; ms_out and launches_out (arrays of
 * FERROX_PHASE_CLASSES, caller-owned host memory) receive the time and the
 * number of launches per class.  Kernel nodes of graphs with conditional nodes
 * are invisible to profilers, so this is the step profilers can see.  ESTATE
 * unless the batch is tuned to (or set to) the graph engine.  Synchronises. */
ferrox_status ferrox_batch_profile_phases(ferrox_batch* b, double* ms_out, int* launches_out);
ferrox_status ferrox_batch_destroy(ferrox_batch* b);

/* Failure-detection check of the bounded device waits: a two-block launch in
 * which one block never reaches the grid barrier, so the other's wait runs out
 * after about `seconds` (<= 5) of SM clock and records the status, which is
 * written to *status_out (FERROX_ETIMEOUT when the limit works).  Synchronises. */
ferrox_status ferrox_check_wait_timeout(double seconds, int* status_out, void* cuda_stream);

/* The carrier exponentials of the residual kernel on their own: ep_dev[i] =
 * e^{u_dev[i]}, em_dev[i] = e^{-u_dev[i]} (device FP64 arrays of n).  The
 * Boltzmann densities n0 e^{phi/V_T} and p0 e^{-phi/V_T} of the carrier model
 * (Sec. II) are formed from this pair; both share one table-driven argument
 * reduction (Tang 1989), within about 1.3 ulp for |u| < 700 and equal to exp()
 * beyond.  n = 0 launches nothing.  Synchronises the stream; FERROX_EINVAL for
 * n < 0 or a null pointer with n > 0. */
ferrox_status ferrox_carrier_exp(const double* u_dev, double* ep_dev, double* em_dev, long long n,
                                 void* cuda_stream);
/* The same pair in double-float arithmetic on the FP32 pipe, as the mixed form's
 * residual evaluates it for |u| <= 70: u_hl_dev holds n arguments as float pairs
 * (u = h + l, 2n floats, 8-byte aligned); ep_dev[i] and em_dev[i] receive the
 * result pairs of e^{+u} and e^{-u} summed in FP64.  About 2^-47 relative for
 * |u| <= 70; outside that range the values are not specified (the residual then
 * uses the FP64 routine).  Synchronises; FERROX_EINVAL for n < 0, a null
 * pointer with n > 0 or a misaligned u_hl_dev. */
ferrox_status ferrox_carrier_exp_df(const float* u_hl_dev, double* ep_dev, double* em_dev, long long n,
                                    void* cuda_stream);
const char* ferrox_batch_last_error(const ferrox_batch* b);

/* ---- learned warm start ------------------------------------------------------------------
 * Not in the paper (the workloads add it).  A small 3-D U-Net (about 80k
 * parameters; BF16 weights and activations, FP32 accumulation on the tensor
 * cores) acts on multigrid level 2 (the fine grid coarsened 2x2x2 twice).  It
 * maps the restricted initial residual of each solve (scaled by its rms) and
 * per-plane material, height and bias features to the restricted error of the
 * initial guess; the prediction is prolongated and added to the guess before
 * the multigrid cycles.  The corrected guess is kept only if its residual norm
 * is below the guess's (or already meets the test); otherwise the solve
 * restarts from the saved guess (stats.nn_rejected counts these).  Multigrid
 * still runs to the residual test, so the network can change the number of
 * cycles, never the converged answer.  Learned steps run the defect-correction
 * form of the solve.
 * Training data are snapshots the solver records in collect mode.
 * Weights: per layer [27][Cin][Cout] FP32 (tap = 9 dz + 3 dy + dx), layers
 * (16,16) (16,16) (16,32) (32,32) (48,16) (16,16); biases [Cout]. */
typedef struct ferrox_nn ferrox_nn; /* opaque */

/* A network for a D x H x W grid (all even) with a store for `capacity`
 * snapshots; the caller supplies the initial weights and biases (host FP32). */
ferrox_status ferrox_nn_create(ferrox_nn** out, int D, int H, int W, int capacity,
                               const float* weights, const float* biases, void* cuda_stream);
/* y_dev[m] = output channel 0 for input x_dev[m][16] (device FP32 arrays). */
ferrox_status ferrox_nn_forward(ferrox_nn* nn, const float* x_dev, float* y_dev);
/* Forward, mean-squared error against t_dev[m], backward: gradients accumulate. */
ferrox_status ferrox_nn_loss_grad(ferrox_nn* nn, const float* x_dev, const float* t_dev,
                                  float* loss_host);
/* Copy weights, biases and accumulated gradients to host arrays (any may be NULL). */
ferrox_status ferrox_nn_params(ferrox_nn* nn, float* w, float* b, float* gw, float* gb);
ferrox_status ferrox_nn_set_params(ferrox_nn* nn, const float* w, const float* b);
/* One Adam update (beta1 0.9, beta2 0.999, eps 1e-8) from the accumulated gradients,
 * which are then cleared. */
ferrox_status ferrox_nn_adam_step(ferrox_nn* nn, double lr);
ferrox_status ferrox_nn_snapshot_count(const ferrox_nn* nn, int* count);
/* `epochs` passes over the stored snapshots, each in a fresh pseudo-random order
 * (fixed seed: repeated calls on the same store repeat), an Adam step every
 * `batch` of them with a step size that decays from lr to lr / 10 (cosine) over
 * the call; loss_per_epoch (host, may be NULL) receives the mean loss of each
 * epoch. */
ferrox_status ferrox_nn_train(ferrox_nn* nn, int epochs, double lr, int batch,
                              float* loss_per_epoch);
ferrox_status ferrox_nn_destroy(ferrox_nn* nn);
const char* ferrox_nn_last_error(const ferrox_nn* nn);
/* Convolution kernels.  use_tensor_memory = 1 (the default) runs every
 * convolution whose grid has an x extent that is a multiple of 8 and a y extent
 * that is a multiple of 16 on the tcgen05 kernel (FP32 accumulators in tensor
 * memory); 0 runs all of them on the mma.sync kernel.  Takes effect for later
 * calls and for graphs captured afterwards.  Returns EINVAL for other values. */
ferrox_status ferrox_nn_use_tensor_memory(ferrox_nn* nn, int use_tensor_memory);
/* After synchronising the network's stream: tc_forward / tc_backward = how many
 * of the 6 forward and 5 adjoint convolutions of one pass run on the tcgen05
 * kernel; fault = 1 if a tcgen05 convolution gave up waiting for its MMAs (about
 * a second; that launch then left its output incomplete), else 0.  Any output
 * may be NULL. */
ferrox_status ferrox_nn_kernel_info(ferrox_nn* nn, int* tc_forward, int* tc_backward, int* fault);
/* Attach a network to a context: mode 0 detaches, 1 records one snapshot per
 * ferrox_step (order 1; the steps then run without a CUDA graph), 2 applies the
 * network before every predictor solve (captured in the step graph).  The
 * network grid must equal the context's level-2 grid. */
ferrox_status ferrox_attach_nn(ferrox_ctx* ctx, ferrox_nn* nn, int mode);

/* Limits of ferrox_tdgl_update_static (sizes of its file-scope scratch array). */
#define FERROX_STATIC_MAX_CELLS 262144
#define FERROX_STATIC_MAX_PLANES 512

/* The explicit TDGL polarization update P <- P + dt f(P, phi) without any
 * device allocation, for callers that cannot allocate device memory: processes
 * held to a fixed device-memory budget, frameworks whose own allocator must own
 * every device byte, and latency-bound loops that cannot afford the device-wide
 * synchronisation that cudaMalloc and cudaFree may imply.  The paper has no
 * counterpart; this is a deployment variant of ferrox_tdgl_update.
 *   geom, dt, v_bottom, v_top: as for ferrox_init_geometry / ferrox_set_bias.
 *   P_dev (in/out) and phi_dev (in): caller-owned device arrays, layout above.
 *   Only the ferroelectric planes of P_dev are written; every other plane keeps
 *   the caller's values.
 * It runs the same fused TDGL kernel, with its scratch (plane table, staging
 * copy of the new P, right-hand side) in one file-scope device array of about
 * 8.1 MB that every GPU loading the library holds until the process exits.
 * Limits: Nx*Ny*Nz <= FERROX_STATIC_MAX_CELLS and Nz <= FERROX_STATIC_MAX_PLANES;
 * larger grids are rejected with FERROX_EINVAL and a message.  No scratch
 * byte is read before the call writes it, so nothing needs clearing between
 * calls.  All calls share the one array: calls whose GPU work overlaps (two
 * streams, or two host threads) race and must be serialised by the caller.
 * The first call on each device looks up the array's device address with
 * that device current.  The plane table is copied from pageable host memory,
 * so the call waits for work already queued on the stream before it returns. */
ferrox_status ferrox_tdgl_update_static(const ferrox_geometry* geom, double dt, double v_bottom,
                                        double v_top, double* P_dev, const double* phi_dev,
                                        void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* FERROX_H */

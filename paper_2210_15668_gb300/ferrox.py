"""Thin ctypes binding of libferrox (include/ferrox.h): argument marshalling only.

Every step of the time step runs in the CUDA library; this module converts
Python dicts to the C structs, passes device pointers of torch tensors and the
current CUDA stream, and turns status codes into exceptions.  There is no CPU
fallback: if the compiled library is missing, loading raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libferrox.so")

FERROX_OK, FERROX_EINVAL, FERROX_ENOMEM, FERROX_ECUDA = 0, 1, 2, 3
FERROX_ENOCONV, FERROX_ENONFINITE, FERROX_ETIMEOUT, FERROX_ESTATE = 4, 5, 6, 7
FP64, MIXED, FP64_DEFECT = 0, 1, 2
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENOCONV", 5: "ENONFINITE",
                6: "ETIMEOUT", 7: "ESTATE"}


class Layer(C.Structure):
    _fields_ = [("kind", C.c_int), ("ncells", C.c_int), ("eps_r", C.c_double),
                ("alpha", C.c_double), ("beta", C.c_double), ("gamma", C.c_double),
                ("alpha_xy", C.c_double), ("beta_xy", C.c_double), ("gamma_xy", C.c_double),
                ("g11", C.c_double), ("g44", C.c_double), ("Gamma", C.c_double),
                ("N_A", C.c_double), ("N_D", C.c_double), ("n_i", C.c_double), ("T", C.c_double),
                ("stats", C.c_int), ("pad", C.c_int), ("m_e", C.c_double), ("m_p", C.c_double),
                ("E_g", C.c_double)]


class Geometry(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("h", C.c_double), ("nlayers", C.c_int),
                ("layers", C.POINTER(Layer)), ("pbc", C.c_int), ("lambda_", C.c_double),
                ("ncomp", C.c_int)]


class Numerics(C.Structure):
    _fields_ = [("dt", C.c_double), ("order", C.c_int), ("tol", C.c_double), ("nu1", C.c_int),
                ("nu2", C.c_int), ("max_cycles", C.c_int), ("precision", C.c_int),
                ("bottom_sweeps", C.c_int), ("guess", C.c_int), ("inner", C.c_int),
                ("nonlinear", C.c_int), ("tdgl_arith", C.c_int)]


class Charge(C.Structure):
    _fields_ = [("Q_int", C.c_double), ("phi_int_avg", C.c_double), ("V_fe", C.c_double),
                ("sigma_top", C.c_double), ("sigma_bot", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("steps", C.c_longlong), ("launches", C.c_longlong), ("solves", C.c_longlong),
                ("cycles", C.c_longlong),
                ("last_cycles", C.c_int), ("last_rel_res", C.c_double), ("status", C.c_int),
                ("vcycles", C.c_longlong), ("nn_rejected", C.c_longlong)]


EXPORTS = ["ferrox_init_geometry", "ferrox_set_bias", "ferrox_solve_poisson", "ferrox_tdgl_update",
           "ferrox_step", "ferrox_charge", "ferrox_sync_stats", "ferrox_clear_status",
           "ferrox_get_state", "ferrox_set_state", "ferrox_fe_planes", "ferrox_get_state_fe",
           "ferrox_set_state_fe", "ferrox_destroy", "ferrox_last_error",
           "ferrox_level_shape", "ferrox_profile_step", "ferrox_profile_step_bytes", "ferrox_qv_sweep", "ferrox_residual",
           "ferrox_tdgl_update_static",
           "ferrox_init_batch", "ferrox_batch_set_bias", "ferrox_batch_solve_poisson",
           "ferrox_batch_step", "ferrox_batch_charge", "ferrox_batch_stats", "ferrox_batch_tuning",
           "ferrox_batch_groups", "ferrox_batch_set_shape", "ferrox_batch_engine", "ferrox_batch_set_engine",
           "ferrox_batch_profile_phases",
           "ferrox_batch_destroy", "ferrox_batch_last_error", "ferrox_check_wait_timeout",
           "ferrox_carrier_exp", "ferrox_carrier_exp_df",
           "ferrox_nn_create", "ferrox_nn_forward", "ferrox_nn_loss_grad", "ferrox_nn_params",
           "ferrox_nn_set_params", "ferrox_nn_adam_step", "ferrox_nn_snapshot_count", "ferrox_nn_train",
           "ferrox_nn_destroy", "ferrox_nn_last_error", "ferrox_nn_use_tensor_memory", "ferrox_nn_kernel_info",
           "ferrox_attach_nn"]

# classes of ferrox_batch_profile_phases, in the header's order
PHASE_CLASSES = ["tdgl", "resid", "decide", "smooth_fine", "smooth_coarse", "transfer", "tail", "other"]

KERNEL_CLASSES = ["tdgl", "resid", "smooth_fine", "smooth_coarse", "restrict", "prolong", "tail",
                  "update", "copy"]

_lib = None


def load(path: str = LIB_PATH):
    """Load libferrox.so and declare its signatures (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libferrox not built ({path} missing): run __graft_entry__.build()")
    lib = C.CDLL(path)
    vp, st = C.c_void_p, C.c_int
    lib.ferrox_init_geometry.argtypes = [C.POINTER(vp), C.POINTER(Geometry), C.POINTER(Numerics),
                                         vp, vp, vp]
    lib.ferrox_set_bias.argtypes = [vp, C.c_double, C.c_double]
    for name in ("ferrox_solve_poisson", "ferrox_tdgl_update", "ferrox_destroy", "ferrox_clear_status"):
        getattr(lib, name).argtypes = [vp]
    lib.ferrox_step.argtypes = [vp, C.c_int]
    lib.ferrox_charge.argtypes = [vp, C.POINTER(Charge)]
    lib.ferrox_sync_stats.argtypes = [vp, C.POINTER(Stats)]
    lib.ferrox_get_state.argtypes = [vp, vp, vp]
    lib.ferrox_set_state.argtypes = [vp, vp, vp]
    lib.ferrox_fe_planes.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    lib.ferrox_get_state_fe.argtypes = [vp, vp, vp]
    lib.ferrox_set_state_fe.argtypes = [vp, vp, vp]
    lib.ferrox_last_error.argtypes = [vp]
    lib.ferrox_last_error.restype = C.c_char_p
    lib.ferrox_level_shape.argtypes = [vp, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                       C.POINTER(C.c_int), C.POINTER(C.c_int)]
    lib.ferrox_profile_step.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_int)]
    lib.ferrox_qv_sweep.argtypes = [vp, C.POINTER(C.c_double), C.c_int, C.c_int, C.POINTER(Charge)]
    lib.ferrox_residual.argtypes = [vp, C.c_int, vp]
    lib.ferrox_profile_step_bytes.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_int),
                                              C.POINTER(C.c_double)]
    lib.ferrox_tdgl_update_static.argtypes = [C.POINTER(Geometry), C.c_double, C.c_double,
                                              C.c_double, vp, vp, vp]
    lib.ferrox_init_batch.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(Geometry),
                                      C.POINTER(Numerics), vp, vp, vp]
    lib.ferrox_batch_set_bias.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    lib.ferrox_batch_solve_poisson.argtypes = [vp]
    lib.ferrox_batch_step.argtypes = [vp, C.c_int]
    lib.ferrox_batch_charge.argtypes = [vp, C.POINTER(Charge)]
    lib.ferrox_batch_stats.argtypes = [vp, C.POINTER(Stats)]
    lib.ferrox_batch_tuning.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]
    lib.ferrox_batch_groups.argtypes = [vp, C.POINTER(C.c_int)]
    lib.ferrox_batch_set_shape.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int]
    lib.ferrox_batch_engine.argtypes = [vp, C.POINTER(C.c_int)]
    lib.ferrox_batch_set_engine.argtypes = [vp, C.c_int]
    lib.ferrox_batch_profile_phases.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_int)]
    lib.ferrox_batch_destroy.argtypes = [vp]
    lib.ferrox_batch_last_error.argtypes = [vp]
    lib.ferrox_batch_last_error.restype = C.c_char_p
    lib.ferrox_check_wait_timeout.argtypes = [C.c_double, C.POINTER(C.c_int), vp]
    lib.ferrox_carrier_exp.argtypes = [vp, vp, vp, C.c_longlong, vp]
    lib.ferrox_carrier_exp_df.argtypes = [vp, vp, vp, C.c_longlong, vp]
    lib.ferrox_attach_nn.argtypes = [vp, vp, C.c_int]
    for name in EXPORTS:
        if name not in ("ferrox_last_error", "ferrox_batch_last_error", "ferrox_nn_last_error"):
            getattr(lib, name).restype = st
    _lib = lib
    return lib


class FerroxError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def make_layers(layers):
    arr = (Layer * len(layers))()
    for q, l in enumerate(layers):
        L = arr[q]
        L.kind, L.ncells, L.eps_r = int(l["kind"]), int(l["ncells"]), float(l["eps_r"])
        for k in ("alpha", "beta", "gamma", "g11", "g44", "Gamma", "N_A", "N_D", "n_i", "T", "m_e",
                  "m_p", "E_g"):
            setattr(L, k, float(l.get(k, 0.0)))
        L.stats = int(l.get("stats", 0))
        for k in ("alpha", "beta", "gamma"):
            setattr(L, k + "_xy", float(l.get(k + "_xy", l.get(k, 0.0))))
    return arr


NEWTON, FIXED_POINT = 0, 1
TDGL_FP64, TDGL_FP32 = 0, 1


def make_numerics(dt, order=1, tol=1e-10, nu1=2, nu2=2, max_cycles=200, precision=FP64,
                  bottom_sweeps=0, guess=0, inner=1, nonlinear=NEWTON, tdgl_arith=TDGL_FP64):
    return Numerics(float(dt), int(order), float(tol), int(nu1), int(nu2), int(max_cycles),
                    int(precision), int(bottom_sweeps), int(guess), int(inner), int(nonlinear),
                    int(tdgl_arith))


def tdgl_update_static(geom, dt, v_bottom, v_top, P, phi, stream=None):
    """P <- P + dt f(P, phi) through the entry point that allocates nothing.

    P, phi: contiguous float64 CUDA tensors (P is updated in place)."""
    import torch
    lib = load()
    layers = make_layers(geom["layers"])
    g = Geometry(geom["nx"], geom["ny"], geom["h"], len(geom["layers"]), layers, geom["pbc"],
                 geom["lam"], geom.get("ncomp", 1))
    st = stream if stream is not None else torch.cuda.current_stream(P.device)
    rc = lib.ferrox_tdgl_update_static(C.byref(g), float(dt), float(v_bottom), float(v_top),
                                       C.c_void_p(P.data_ptr()), C.c_void_p(phi.data_ptr()),
                                       C.c_void_p(st.cuda_stream))
    if rc != FERROX_OK:
        raise FerroxError(rc, lib.ferrox_last_error(None).decode())


class Device:
    """One device stack on the current GPU: caller-owned torch state + a libferrox context.

    geom: dict from paper_2210_15668_gb300.inputs.make_geometry; P0: (ncomp, Nz, Ny, Nx) array.
    """

    def __init__(self, geom, P0, numerics=None, phi0=None, stream=None, device="cuda:0"):
        import torch
        self.lib = load()
        self.torch = torch
        self.geom = geom
        nz = sum(l["ncells"] for l in geom["layers"])
        self.shape = (nz, geom["ny"], geom["nx"])
        self.ncomp = geom.get("ncomp", 1)
        self.P = torch.as_tensor(np.asarray(P0, dtype=np.float64), device=device).contiguous().clone()
        if phi0 is None:
            self.phi = torch.zeros(self.shape, dtype=torch.float64, device=device)
        else:
            self.phi = torch.as_tensor(np.asarray(phi0, dtype=np.float64), device=device).contiguous().clone()
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.P.device)
        self._layers = make_layers(geom["layers"])
        g = Geometry(geom["nx"], geom["ny"], geom["h"], len(geom["layers"]), self._layers,
                     geom["pbc"], geom["lam"], self.ncomp)
        self.numerics = numerics if numerics is not None else make_numerics(4e-13)
        self.ctx = C.c_void_p()
        rc = self.lib.ferrox_init_geometry(C.byref(self.ctx), C.byref(g), C.byref(self.numerics),
                                           C.c_void_p(self.P.data_ptr()),
                                           C.c_void_p(self.phi.data_ptr()),
                                           C.c_void_p(self.stream.cuda_stream))
        if rc != FERROX_OK:
            raise FerroxError(rc, self.lib.ferrox_last_error(None).decode())

    def _ck(self, rc):
        if rc != FERROX_OK:
            raise FerroxError(rc, self.lib.ferrox_last_error(self.ctx).decode())

    def set_bias(self, v_bottom, v_top):
        self._ck(self.lib.ferrox_set_bias(self.ctx, float(v_bottom), float(v_top)))

    def solve_poisson(self):
        self._ck(self.lib.ferrox_solve_poisson(self.ctx))

    def tdgl_update(self):
        self._ck(self.lib.ferrox_tdgl_update(self.ctx))

    def step(self, n=1):
        self._ck(self.lib.ferrox_step(self.ctx, int(n)))

    def charge(self):
        out = Charge()
        self._ck(self.lib.ferrox_charge(self.ctx, C.byref(out)))
        return {k: getattr(out, k) for k, _ in Charge._fields_}

    def stats(self, check=True):
        out = Stats()
        rc = self.lib.ferrox_sync_stats(self.ctx, C.byref(out))
        if check:
            self._ck(rc)
        return {k: getattr(out, k) for k, _ in Stats._fields_}

    def clear_status(self):
        self._ck(self.lib.ferrox_clear_status(self.ctx))

    def get_state(self, P_host=None, phi_host=None):
        """Copy the state into host numpy arrays (allocated if not given); synchronises."""
        P_host = np.empty((self.ncomp,) + self.shape) if P_host is None else P_host
        phi_host = np.empty(self.shape) if phi_host is None else phi_host
        self._ck(self.lib.ferrox_get_state(self.ctx, C.c_void_p(P_host.ctypes.data),
                                           C.c_void_p(phi_host.ctypes.data)))
        return P_host, phi_host

    def set_state(self, P_host=None, phi_host=None):
        """Asynchronous copy from host arrays (keep them alive until the stream syncs)."""
        self._keep = (P_host, phi_host)
        pp = C.c_void_p(P_host.ctypes.data) if P_host is not None else None
        fp = C.c_void_p(phi_host.ctypes.data) if phi_host is not None else None
        self._ck(self.lib.ferrox_set_state(self.ctx, pp, fp))

    def fe_planes(self):
        """(fe_lo, fe_hi): the planes of the ferroelectric film (P is zero elsewhere)."""
        lo, hi = C.c_int(), C.c_int()
        self._ck(self.lib.ferrox_fe_planes(self.ctx, C.byref(lo), C.byref(hi)))
        return lo.value, hi.value

    def get_state_fe(self, P_fe_host=None, phi_host=None):
        """Like get_state with P restricted to the film: [ncomp][fe_hi-fe_lo+1][ny][nx]."""
        lo, hi = self.fe_planes()
        P_fe_host = np.empty((self.ncomp, hi - lo + 1) + self.shape[1:]) if P_fe_host is None else P_fe_host
        phi_host = np.empty(self.shape) if phi_host is None else phi_host
        self._ck(self.lib.ferrox_get_state_fe(self.ctx, C.c_void_p(P_fe_host.ctypes.data),
                                              C.c_void_p(phi_host.ctypes.data)))
        return P_fe_host, phi_host

    def set_state_fe(self, P_fe_host=None, phi_host=None):
        """Asynchronous copy of the film's P and of phi (keep the arrays alive until the stream syncs)."""
        self._keep = (P_fe_host, phi_host)
        pp = C.c_void_p(P_fe_host.ctypes.data) if P_fe_host is not None else None
        fp = C.c_void_p(phi_host.ctypes.data) if phi_host is not None else None
        self._ck(self.lib.ferrox_set_state_fe(self.ctx, pp, fp))

    def residual(self, double_float=False):
        """r = b + rho(phi) - A phi of the current state (scaled by h^2/eps0), float64
        [Nz][Ny][Nx], in FP64 or in the mixed form's double-float arithmetic."""
        import numpy as np
        nz = sum(int(l["ncells"]) for l in self.geom["layers"])
        out = np.empty((nz, self.geom["ny"], self.geom["nx"]), dtype=np.float64)
        self._ck(self.lib.ferrox_residual(self.ctx, 1 if double_float else 0,
                                          C.c_void_p(out.ctypes.data)))
        return out

    def qv_sweep(self, v_app, steps_per_point):
        """Triangular-wave (or any) Q-V protocol run natively: a list of charge
        records {Q_int, phi_int_avg, V_fe, sigma_top, sigma_bot}, one per bias point."""
        v = (C.c_double * len(v_app))(*[float(x) for x in v_app])
        out = (Charge * len(v_app))()
        self._ck(self.lib.ferrox_qv_sweep(self.ctx, v, len(v_app), int(steps_per_point), out))
        return [{k: getattr(o, k) for k, _ in Charge._fields_} for o in out]

    def profile_step(self, with_bytes=False):
        """One event-timed eager step: {kernel class: (total ms, launches)}, or with
        with_bytes {kernel class: (total ms, launches, algorithmic bytes)}."""
        n = len(KERNEL_CLASSES)
        ms = (C.c_double * n)()
        cnt = (C.c_int * n)()
        by = (C.c_double * n)()
        self._ck(self.lib.ferrox_profile_step_bytes(self.ctx, ms, cnt, by))
        if with_bytes:
            return {KERNEL_CLASSES[k]: (ms[k], cnt[k], by[k]) for k in range(n)}
        return {KERNEL_CLASSES[k]: (ms[k], cnt[k]) for k in range(n)}

    def attach_nn(self, net, mode):
        """mode 0: detach; 1: collect snapshots each step; 2: apply before each solve."""
        self._ck(self.lib.ferrox_attach_nn(self.ctx, net.ctx if net is not None else None, int(mode)))

    def levels(self):
        n = C.c_int()
        nx, ny, nz = C.c_int(), C.c_int(), C.c_int()
        self.lib.ferrox_level_shape(self.ctx, 0, C.byref(nx), C.byref(ny), C.byref(nz), C.byref(n))
        out = []
        for l in range(n.value):
            self.lib.ferrox_level_shape(self.ctx, l, C.byref(nx), C.byref(ny), C.byref(nz), None)
            out.append((nx.value, ny.value, nz.value))
        return out

    def close(self):
        if self.ctx:
            self.lib.ferrox_destroy(self.ctx)
            self.ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """n independent device stacks advanced together (one persistent launch per call, or a
    CUDA graph of per-phase launches: the autotuner picks).

    geoms: list of geometry dicts (ncomp = 1); P0s: list of (1, Nz, Ny, Nx) arrays.
    The state lives in two packed torch tensors (instances back to back)."""

    def __init__(self, geoms, P0s, numerics, stream=None, device="cuda:0"):
        import torch
        self.lib = load()
        self.geoms = geoms
        self.shapes = [(sum(l["ncells"] for l in g["layers"]), g["ny"], g["nx"]) for g in geoms]
        self.sizes = [int(np.prod(s)) for s in self.shapes]
        self.offsets = np.concatenate([[0], np.cumsum(self.sizes)]).astype(np.int64)
        flat = np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in P0s])
        self.P = torch.as_tensor(flat, device=device).contiguous().clone()
        self.phi = torch.zeros_like(self.P)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.P.device)
        self._layers = [make_layers(g["layers"]) for g in geoms]
        garr = (Geometry * len(geoms))()
        for q, g in enumerate(geoms):
            garr[q] = Geometry(g["nx"], g["ny"], g["h"], len(g["layers"]), self._layers[q], g["pbc"],
                               g["lam"], 1)
        self._garr = garr
        self.numerics = numerics
        self.ctx = C.c_void_p()
        rc = self.lib.ferrox_init_batch(C.byref(self.ctx), len(geoms), garr, C.byref(numerics),
                                        C.c_void_p(self.P.data_ptr()), C.c_void_p(self.phi.data_ptr()),
                                        C.c_void_p(self.stream.cuda_stream))
        if rc != FERROX_OK:
            raise FerroxError(rc, self.lib.ferrox_batch_last_error(None).decode())

    def _ck(self, rc):
        if rc != FERROX_OK:
            raise FerroxError(rc, self.lib.ferrox_batch_last_error(self.ctx).decode())

    def set_bias(self, v_bottom, v_top):
        n = len(self.geoms)
        vb = (C.c_double * n)(*[float(v) for v in np.broadcast_to(v_bottom, n)])
        vt = (C.c_double * n)(*[float(v) for v in np.broadcast_to(v_top, n)])
        self._ck(self.lib.ferrox_batch_set_bias(self.ctx, vb, vt))

    def solve_poisson(self):
        self._ck(self.lib.ferrox_batch_solve_poisson(self.ctx))

    def step(self, n=1):
        self._ck(self.lib.ferrox_batch_step(self.ctx, int(n)))

    def stats(self, check=True):
        n = len(self.geoms)
        out = (Stats * n)()
        rc = self.lib.ferrox_batch_stats(self.ctx, out)
        if check:
            self._ck(rc)
        return [{k: getattr(o, k) for k, _ in Stats._fields_} for o in out]

    def charge(self):
        n = len(self.geoms)
        out = (Charge * n)()
        self._ck(self.lib.ferrox_batch_charge(self.ctx, out))
        return [{k: getattr(o, k) for k, _ in Charge._fields_} for o in out]

    def tuning(self):
        t, r, b = C.c_int(), C.c_int(), C.c_int()
        rc = self.lib.ferrox_batch_tuning(self.ctx, C.byref(t), C.byref(r), C.byref(b))
        g = C.c_int()
        self.lib.ferrox_batch_groups(self.ctx, C.byref(g))
        e = C.c_int()
        self.lib.ferrox_batch_engine(self.ctx, C.byref(e))
        return dict(threads=t.value, rows_per_unit=r.value, blocks=b.value, groups=g.value,
                    engine=e.value, tuned=rc == FERROX_OK)

    def set_engine(self, engine):
        """0: one persistent launch; 1: the graph of per-phase launches (same results)."""
        self._ck(self.lib.ferrox_batch_set_engine(self.ctx, int(engine)))

    def profile_phases(self):
        """One time step with the graph engine's kernels launched one by one (the state
        advances as step(1) would); {class: (ms, launches)} from CUDA events."""
        n = len(PHASE_CLASSES)
        ms = (C.c_double * n)()
        nl = (C.c_int * n)()
        self._ck(self.lib.ferrox_batch_profile_phases(self.ctx, ms, nl))
        return {k: (ms[q], nl[q]) for q, k in enumerate(PHASE_CLASSES)}

    def set_shape(self, threads, rows_per_unit, ctas_per_sm, grouped):
        """Fix the launch shape instead of autotuning it (same results, other speed)."""
        self._ck(self.lib.ferrox_batch_set_shape(self.ctx, int(threads), int(rows_per_unit),
                                                 int(ctas_per_sm), int(grouped)))

    def state(self, i):
        """(P, phi) of instance i as numpy arrays (synchronises)."""
        import torch
        torch.cuda.synchronize()
        a, b = self.offsets[i], self.offsets[i + 1]
        shp = self.shapes[i]
        return (self.P[a:b].cpu().numpy().reshape((1,) + shp), self.phi[a:b].cpu().numpy().reshape(shp))

    def close(self):
        if self.ctx:
            self.lib.ferrox_batch_destroy(self.ctx)
            self.ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def check_wait_timeout(seconds=0.2, stream=None):
    """Run the bounded-wait check; returns the status the device recorded."""
    import torch
    lib = load()
    st = stream if stream is not None else torch.cuda.current_stream()
    out = C.c_int(-1)
    rc = lib.ferrox_check_wait_timeout(float(seconds), C.byref(out), C.c_void_p(st.cuda_stream))
    if rc != FERROX_OK:
        raise FerroxError(rc, lib.ferrox_batch_last_error(None).decode())
    return out.value


def carrier_exp(u, stream=None):
    """(e^u, e^-u) of a CUDA FP64 tensor, by the residual kernel's carrier routine."""
    import torch
    lib = load()
    if not (u.is_cuda and u.dtype == torch.float64):
        raise TypeError("u must be a CUDA float64 tensor")
    u = u.contiguous()
    st = stream if stream is not None else torch.cuda.current_stream()
    ep = torch.empty_like(u)
    em = torch.empty_like(u)
    rc = lib.ferrox_carrier_exp(C.c_void_p(u.data_ptr()), C.c_void_p(ep.data_ptr()),
                                C.c_void_p(em.data_ptr()), u.numel(), C.c_void_p(st.cuda_stream))
    if rc != FERROX_OK:
        raise FerroxError(rc, lib.ferrox_batch_last_error(None).decode())
    return ep, em


def carrier_exp_df(u_hl, stream=None):
    """(e^u, e^-u) in double-float arithmetic for arguments given as float pairs: u_hl
    a CUDA float32 tensor [n, 2] (h, l); the result pairs are returned summed in FP64."""
    import torch
    lib = load()
    if not (u_hl.is_cuda and u_hl.dtype == torch.float32 and u_hl.dim() == 2 and u_hl.shape[1] == 2):
        raise TypeError("u_hl must be a CUDA float32 tensor of shape [n, 2]")
    u_hl = u_hl.contiguous()
    st = stream if stream is not None else torch.cuda.current_stream()
    n = u_hl.shape[0]
    ep = torch.empty(n, dtype=torch.float64, device=u_hl.device)
    em = torch.empty(n, dtype=torch.float64, device=u_hl.device)
    rc = lib.ferrox_carrier_exp_df(C.c_void_p(u_hl.data_ptr()), C.c_void_p(ep.data_ptr()),
                                   C.c_void_p(em.data_ptr()), C.c_longlong(n), C.c_void_p(st.cuda_stream))
    if rc != FERROX_OK:
        raise FerroxError(rc, lib.ferrox_batch_last_error(None).decode())
    return ep, em


NN_LAYERS = [(16, 16), (16, 16), (16, 32), (32, 32), (48, 16), (16, 16)]


def nn_param_sizes():
    return [27 * ci * co for ci, co in NN_LAYERS], [co for _, co in NN_LAYERS]


def nn_init_params(seed):
    """He-normal initial weights (math layout [27][Cin][Cout] per layer) and zero biases."""
    rng = np.random.default_rng(seed)
    ws = [rng.standard_normal((27, ci, co)) * np.sqrt(2.0 / (27 * ci)) for ci, co in NN_LAYERS]
    bs = [np.zeros(co) for _, co in NN_LAYERS]
    return ws, bs


class NN:
    """The learned warm-start network on one grid (channels-last, 16 input channels)."""

    def __init__(self, D, H, W, capacity=0, params=None, seed=0, stream=None):
        import torch
        self.lib = load()
        lib = self.lib
        if not getattr(lib, "_nn_declared", False):
            vp = C.c_void_p
            fp = C.POINTER(C.c_float)
            lib.ferrox_nn_create.argtypes = [C.POINTER(vp), C.c_int, C.c_int, C.c_int, C.c_int, fp, fp, vp]
            lib.ferrox_nn_forward.argtypes = [vp, vp, vp]
            lib.ferrox_nn_loss_grad.argtypes = [vp, vp, vp, fp]
            lib.ferrox_nn_params.argtypes = [vp, fp, fp, fp, fp]
            lib.ferrox_nn_set_params.argtypes = [vp, fp, fp]
            lib.ferrox_nn_adam_step.argtypes = [vp, C.c_double]
            lib.ferrox_nn_snapshot_count.argtypes = [vp, C.POINTER(C.c_int)]
            lib.ferrox_nn_train.argtypes = [vp, C.c_int, C.c_double, C.c_int, fp]
            lib.ferrox_nn_destroy.argtypes = [vp]
            lib.ferrox_nn_last_error.argtypes = [vp]
            lib.ferrox_nn_last_error.restype = C.c_char_p
            ip = C.POINTER(C.c_int)
            lib.ferrox_nn_use_tensor_memory.argtypes = [vp, C.c_int]
            lib.ferrox_nn_kernel_info.argtypes = [vp, ip, ip, ip]
            for n in ("ferrox_nn_create", "ferrox_nn_forward", "ferrox_nn_loss_grad", "ferrox_nn_params",
                      "ferrox_nn_set_params", "ferrox_nn_adam_step", "ferrox_nn_snapshot_count",
                      "ferrox_nn_train", "ferrox_nn_destroy", "ferrox_nn_use_tensor_memory",
                      "ferrox_nn_kernel_info"):
                getattr(lib, n).restype = C.c_int
            lib._nn_declared = True
        self.shape = (D, H, W)
        self.M = D * H * W
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        ws, bs = params if params is not None else nn_init_params(seed)
        wflat = np.concatenate([np.asarray(w, np.float32).ravel() for w in ws])
        bflat = np.concatenate([np.asarray(b, np.float32).ravel() for b in bs])
        self.ctx = C.c_void_p()
        rc = lib.ferrox_nn_create(C.byref(self.ctx), D, H, W, capacity,
                                  wflat.ctypes.data_as(C.POINTER(C.c_float)),
                                  bflat.ctypes.data_as(C.POINTER(C.c_float)), C.c_void_p(self.stream.cuda_stream))
        if rc != FERROX_OK:
            raise FerroxError(rc, lib.ferrox_nn_last_error(None).decode())

    def _ck(self, rc):
        if rc != FERROX_OK:
            raise FerroxError(rc, self.lib.ferrox_nn_last_error(self.ctx).decode())

    def forward(self, x):
        """x: float32 CUDA tensor [M, 16] -> float32 CUDA tensor [M] (output channel 0)."""
        import torch
        y = torch.empty(self.M, dtype=torch.float32, device=x.device)
        self._ck(self.lib.ferrox_nn_forward(self.ctx, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr())))
        return y

    def loss_grad(self, x, t):
        out = C.c_float()
        self._ck(self.lib.ferrox_nn_loss_grad(self.ctx, C.c_void_p(x.data_ptr()), C.c_void_p(t.data_ptr()),
                                              C.byref(out)))
        return out.value

    def params(self):
        nw, nb = nn_param_sizes()
        w = np.empty(sum(nw), np.float32); b = np.empty(sum(nb), np.float32)
        gw = np.empty(sum(nw), np.float32); gb = np.empty(sum(nb), np.float32)
        fp = C.POINTER(C.c_float)
        self._ck(self.lib.ferrox_nn_params(self.ctx, w.ctypes.data_as(fp), b.ctypes.data_as(fp),
                                           gw.ctypes.data_as(fp), gb.ctypes.data_as(fp)))
        return _split(w, nw), _split(b, nb), _split(gw, nw), _split(gb, nb)

    def set_params(self, ws, bs):
        fp = C.POINTER(C.c_float)
        wf = np.concatenate([np.asarray(w, np.float32).ravel() for w in ws])
        bf = np.concatenate([np.asarray(b, np.float32).ravel() for b in bs])
        self._ck(self.lib.ferrox_nn_set_params(self.ctx, wf.ctypes.data_as(fp), bf.ctypes.data_as(fp)))

    def use_tensor_memory(self, on=True):
        """Run the convolutions on the tcgen05 kernel where the grid allows (default), or
        all of them on the mma.sync kernel."""
        self._ck(self.lib.ferrox_nn_use_tensor_memory(self.ctx, 1 if on else 0))

    def kernel_info(self):
        """Number of forward / adjoint convolutions on the tcgen05 kernel, and its fault flag."""
        f, b, flt = C.c_int(), C.c_int(), C.c_int()
        self._ck(self.lib.ferrox_nn_kernel_info(self.ctx, C.byref(f), C.byref(b), C.byref(flt)))
        return {"tc_forward": f.value, "tc_backward": b.value, "fault": flt.value}

    def adam_step(self, lr):
        self._ck(self.lib.ferrox_nn_adam_step(self.ctx, float(lr)))

    def snapshot_count(self):
        n = C.c_int()
        self._ck(self.lib.ferrox_nn_snapshot_count(self.ctx, C.byref(n)))
        return n.value

    def train(self, epochs, lr, batch=8):
        losses = np.zeros(max(epochs, 1), np.float32)
        self._ck(self.lib.ferrox_nn_train(self.ctx, int(epochs), float(lr), int(batch),
                                          losses.ctypes.data_as(C.POINTER(C.c_float))))
        return losses[:epochs]

    def close(self):
        if self.ctx:
            self.lib.ferrox_nn_destroy(self.ctx)
            self.ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _split(flat, sizes):
    out, o = [], 0
    for n in sizes:
        out.append(flat[o:o + n])
        o += n
    return out

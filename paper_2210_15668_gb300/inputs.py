"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module holds data only: the layer stacks of the device workloads and the
seeded random initial polarization.  It contains none of the method's
arithmetic (no operator, no force, no solver), so the oracle and the CUDA path
can both take their inputs from here without sharing any computation.

Materials follow the paper's Table 1 (HZO ferroelectric, SiO2 / Al2O3
dielectrics, Si semiconductor).  The gradient coefficient of the device
workloads is g = 1e-10 (the value the workloads are specified with; Table 1
prints 1e-9 and both are accepted by the code).  Layers are listed bottom to
top; the ferroelectric sits next to the top electrode (Fig. 1a, MFISM with HZO
on top).

Random initial polarization: i.i.d. uniform in [-A, A] C/m^2 on ferroelectric
cells, zero elsewhere (Methods, "Numerical Approach": P initialised with
uniformly distributed random numbers; the supplement uses [-0.002, 0.002]).
The generator is numpy's PCG64, which gives the same stream on every platform.
"""
from __future__ import annotations

import numpy as np

FE, DE, SC = 0, 1, 2

# Table 1: HZO Landau coefficients (SI), permittivities, kinetic coefficient.
HZO = dict(alpha=-2.5e9, beta=6.0e10, gamma=1.5e11, eps_r=24.0, Gamma=100.0)
EPS_SIO2 = 3.9
EPS_AL2O3 = 10.0
EPS_SI = 11.7
H_DEFAULT = 0.5e-9
DT_DEFAULT = 4.0e-13
LAMBDA_DEFAULT = 3.0e-9

PBC_FREE, PBC_ZERO, PBC_LAMBDA = 0, 1, 2


def fe_layer(ncells, g=1e-10, **over):
    d = dict(kind=FE, ncells=int(ncells), eps_r=HZO["eps_r"], alpha=HZO["alpha"],
             beta=HZO["beta"], gamma=HZO["gamma"], g11=g, g44=g, Gamma=HZO["Gamma"],
             N_A=0.0, N_D=0.0, n_i=0.0, T=300.0)
    d.update(over)
    return d


def de_layer(ncells, eps_r=EPS_SIO2):
    return dict(kind=DE, ncells=int(ncells), eps_r=float(eps_r), alpha=0.0, beta=0.0,
                gamma=0.0, g11=0.0, g44=0.0, Gamma=0.0, N_A=0.0, N_D=0.0, n_i=0.0, T=300.0)


# Carrier statistics of a semiconductor layer, and Si data for the Fermi-Dirac model:
# effective masses from the paper's Table 1; the band gap (not in the paper) is the
# usual 300 K value for Si.
STATS_BOLTZMANN, STATS_FERMI_DIRAC = 0, 1
SI_ME, SI_MP, SI_EG = 1.08, 0.81, 1.12


def sc_layer(ncells, N_A=1e24, N_D=0.0, n_i=1e16, T=300.0, eps_r=EPS_SI, stats=STATS_BOLTZMANN,
             m_e=SI_ME, m_p=SI_MP, E_g=SI_EG):
    return dict(kind=SC, ncells=int(ncells), eps_r=float(eps_r), alpha=0.0, beta=0.0,
                gamma=0.0, g11=0.0, g44=0.0, Gamma=0.0, N_A=float(N_A), N_D=float(N_D),
                n_i=float(n_i), T=float(T), stats=int(stats), m_e=float(m_e), m_p=float(m_p),
                E_g=float(E_g))


def make_geometry(nx, ny, layers, h=H_DEFAULT, pbc=PBC_LAMBDA, lam=LAMBDA_DEFAULT, ncomp=1):
    """A geometry record: lateral cells, spacing, layer list (bottom to top), P boundary."""
    return dict(nx=int(nx), ny=int(ny), h=float(h), layers=[dict(l) for l in layers],
                pbc=int(pbc), lam=float(lam), ncomp=int(ncomp))


def nz_of(geom):
    return sum(l["ncells"] for l in geom["layers"])


def fe_plane_mask(geom):
    """Boolean per z-plane: True where the plane belongs to a ferroelectric layer."""
    m = []
    for l in geom["layers"]:
        m += [l["kind"] == FE] * l["ncells"]
    return np.array(m, dtype=bool)


def random_polarization(geom, seed, amp=1e-3, ncomp=None):
    """P[c][z][y][x] float64: U[-amp, amp] on ferroelectric cells, 0 elsewhere."""
    ncomp = geom["ncomp"] if ncomp is None else ncomp
    nz = nz_of(geom)
    rng = np.random.default_rng(seed)
    P = rng.uniform(-amp, amp, size=(ncomp, nz, geom["ny"], geom["nx"]))
    P[:, ~fe_plane_mask(geom)] = 0.0
    return np.ascontiguousarray(P)


def random_polarization_y_uniform(geom, seed, amp=1e-3, ncomp=None):
    """The paper's 2-D setting (Results, MFIM): P uniform along y, U[-amp, amp] in the
    x-z plane of ferroelectric cells, zero elsewhere; P[c][z][y][x] float64."""
    ncomp = geom["ncomp"] if ncomp is None else ncomp
    nz = nz_of(geom)
    rng = np.random.default_rng(seed)
    xz = rng.uniform(-amp, amp, size=(ncomp, nz, 1, geom["nx"]))
    P = np.repeat(xz, geom["ny"], axis=2)
    P[:, ~fe_plane_mask(geom)] = 0.0
    return np.ascontiguousarray(P)


def triangle_wave(v_max, points_per_quarter, sweeps=1):
    """Bias points of the triangular voltage protocol of the Q-V characteristics
    (Results, MFIM): 0 -> +v_max -> 0 -> -v_max -> 0, repeated `sweeps` times, in
    steps of v_max / points_per_quarter (each turning point visited once)."""
    q = int(points_per_quarter)
    up = np.arange(1, q + 1) / q
    period = np.concatenate([up, 1.0 - up, -up, -1.0 + up]) * float(v_max)
    return list(np.tile(period, int(sweeps)))


# --- the device workloads -------------------------------------------------------------

def mfim_stack(nz, n_fe=10, eps_de=EPS_SIO2, g=1e-10):
    """Metal / DE / FE (top n_fe planes) / metal."""
    return [de_layer(nz - n_fe, eps_de), fe_layer(n_fe, g=g)]


def mfism_stack(nz, n_fe=10, n_ox=2, N_A=1e24, n_i=1e16, T=300.0, g=1e-10):
    """Metal / p-Si / SiO2 / FE / metal, bottom to top."""
    return [sc_layer(nz - n_fe - n_ox, N_A=N_A, n_i=n_i, T=T), de_layer(n_ox, EPS_SIO2),
            fe_layer(n_fe, g=g)]


def mfim_small():
    """64x64x16 MFIM, h = 0.5 nm: 3 nm SiO2 under 5 nm HZO; 0.5 V on top; seed 0; 100 steps."""
    return dict(name="mfim_64x64x16", geom=make_geometry(64, 64, mfim_stack(16)), seed=0,
                v_bottom=0.0, v_top=0.5, steps=100, dt=DT_DEFAULT, order=1, precision=0)


def mfim_sweep():
    """256x256x32 MFIM, seed 1; Q-V sweep over linspace(-2, 2, 41), 500 steps per point."""
    return dict(name="mfim_256x256x32", geom=make_geometry(256, 256, mfim_stack(32)), seed=1,
                v_bottom=0.0, v_top=-2.0, sweep=list(np.linspace(-2.0, 2.0, 41)),
                steps_per_point=500, dt=DT_DEFAULT, order=1, precision=0)


def mfism_mixed(nx=256, nz=64):
    """256x256x64 MFISM (p-Si N_A = 1e24, n_i = 1e16, 300 K), seed 2, V = 0, 200 steps."""
    return dict(name=f"mfism_{nx}x{nx}x{nz}", geom=make_geometry(nx, nx, mfism_stack(nz)), seed=2,
                v_bottom=0.0, v_top=0.0, steps=200, dt=DT_DEFAULT, order=1, precision=1)


def batch_sweep(n=64, seed=3, sizes=(32, 48, 64, 96, 128), nz=16):
    """n MFIM instances, lateral size drawn from `sizes`, bias U[-2, 2] V, P seeded per instance."""
    rng = np.random.default_rng(seed)
    lat = rng.choice(np.array(sizes), size=n)
    v = rng.uniform(-2.0, 2.0, size=n)
    inst = []
    for i in range(n):
        inst.append(dict(geom=make_geometry(int(lat[i]), int(lat[i]), mfim_stack(nz)),
                         v_top=float(v[i]), v_bottom=0.0, seed=int(seed) * 1000 + i))
    return inst


def mfism_large():
    """512x512x128 MFISM, seed 5, V = 0, 100 steps."""
    return dict(name="mfism_512x512x128", geom=make_geometry(512, 512, mfism_stack(128)), seed=5,
                v_bottom=0.0, v_top=0.0, steps=100, dt=DT_DEFAULT, order=1, precision=1)


def convergence_cube(n, stats=STATS_FERMI_DIRAC, eps_de=EPS_SIO2):
    """The convergence-study problem of the Numerical Validation section: a 32 nm cube
    of n^3 cells, bottom 25% undoped Si (Fermi-Dirac carriers, the paper's model), 25%
    dielectric (SiO2), top 50% ferroelectric with the parameter table's g = 1e-9,
    lambda = 3 nm; Phi = 0 on both faces is the caller's bias."""
    q = n // 4
    layers = [sc_layer(q, N_A=0.0, stats=stats), de_layer(q, eps_de), fe_layer(2 * q, g=1e-9)]
    return make_geometry(n, n, layers, h=32e-9 / n, pbc=PBC_LAMBDA, lam=3e-9)


def gaussian_bump(geom, amp=0.002, s1=5e-9, s2=2e-9, z0=24e-9):
    """P = amp exp(-(x^2 + y^2)/(2 s1^2) - (z - z0)^2/(2 s2^2)) on ferroelectric cells,
    x, y measured from the centre of the periodic cross-section, z from the bottom."""
    n, h = geom["nx"], geom["h"]
    nz = nz_of(geom)
    c = (np.arange(n) + 0.5) * h - n * h / 2
    cy = (np.arange(geom["ny"]) + 0.5) * h - geom["ny"] * h / 2
    z = (np.arange(nz) + 0.5) * h
    Z, Y, X = np.meshgrid(z, cy, c, indexing="ij")
    P = amp * np.exp(-(X ** 2 + Y ** 2) / (2 * s1 ** 2) - (Z - z0) ** 2 / (2 * s2 ** 2))
    P[~fe_plane_mask(geom)] = 0.0
    return np.ascontiguousarray(P[None])

"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test checks the oracle against something other than itself: a closed form
(layered stack, depolarization field of the Results section, Landau equilibrium,
tanh domain wall, integrator amplification factors, Debye screening), a brute-force
dense solve, or the convergence rates of Table 2.  Each is chosen so that a
plausible slip in the oracle (a dropped term, a flipped sign, a wrong weight or
index) fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import poisson, tdgl, carriers, diagnostics
from oracle.stack import EPS0, Q_E, K_B
from paper_2210_15668_gb300 import inputs as I


def layered(nx, ny, n_de, n_fe, eps_de=3.9, pbc=I.PBC_FREE, h=0.5e-9, **fe):
    return I.make_geometry(nx, ny, [I.de_layer(n_de, eps_de), I.fe_layer(n_fe, **fe)], h=h, pbc=pbc)


def uniform_P(geom, value, ncomp=1):
    nz = I.nz_of(geom)
    P = np.zeros((ncomp, nz, geom["ny"], geom["nx"]))
    P[-1, I.fe_plane_mask(geom)] = value
    return P


# ---------------------------------------------------------------- Poisson operator ----

@pytest.mark.parametrize("V,Pval", [(0.5, 0.2), (0.0, 0.2), (-1.3, -0.05), (2.0, 0.0)])
def test_layered_stack_closed_form(V, Pval):
    """Metal/DE/FE/metal with x-y uniform P: Phi is piecewise linear with
    D = (-V + P t_fe/eps_fe)/(t_fe/eps_fe + t_de/eps_de); the scheme must hit it at
    every cell centre, and dPhi/dz in the FE must equal -E_fe."""
    h = 0.5e-9
    n_de, n_fe = 6, 10
    g = layered(4, 3, n_de, n_fe)
    pl = oracle.planes(g)
    P = uniform_P(g, Pval)
    phi = poisson.solve_linear(P, pl, h, 0.0, V)
    e_de, e_fe = EPS0 * 3.9, EPS0 * 24.0
    t_de, t_fe = n_de * h, n_fe * h
    D = (-V + Pval * t_fe / e_fe) / (t_fe / e_fe + t_de / e_de)
    z = (np.arange(n_de + n_fe) + 0.5) * h
    exact = np.where(z < t_de, -D / e_de * z,
                     -D / e_de * t_de - (D - Pval) / e_fe * (z - t_de))
    err = np.abs(phi - exact[:, None, None]).max()
    assert err <= 1e-13 * max(1.0, np.abs(exact).max())
    E_fe = (D - Pval) / e_fe
    dz = tdgl.dphi_dz(phi, P, pl, h, 0.0, V)
    fe = pl["fe"]
    assert np.abs(dz[fe] + E_fe).max() <= 1e-12 * max(abs(E_fe), 1.0)
    if V == 0.0:
        # depolarization field of the FE/DE series stack at zero bias (Results, MFIM):
        E_dep = -Pval / (EPS0 * (24.0 + 3.9 * t_fe / t_de))
        assert abs(E_fe - E_dep) <= 1e-12 * abs(E_dep)
    d = diagnostics.charges(phi, P, pl, g, 0.0, V)
    assert abs(d["Q_int"] + D) <= 1e-12 * max(abs(D), 1e-3)
    assert abs(d["sigma_top"] + D) <= 1e-12 * max(abs(D), 1e-3)
    assert abs(d["sigma_bot"] - D) <= 1e-12 * max(abs(D), 1e-3)
    phi_int = -D / e_de * t_de
    assert abs(d["V_fe"] - (V - phi_int)) <= 1e-12 * max(1.0, abs(V))


def test_linear_capacitor_charge():
    """All-dielectric stack: sigma_top = eps V / L exactly, and Phi is linear."""
    h = 0.5e-9
    g = I.make_geometry(5, 4, [I.de_layer(12, 10.0)], h=h)
    pl = oracle.planes(g)
    P = np.zeros((1, 12, 4, 5))
    V = 0.7
    phi = poisson.solve_linear(P, pl, h, 0.0, V)
    L = 12 * h
    z = (np.arange(12) + 0.5) * h
    assert np.abs(phi - (V * z / L)[:, None, None]).max() < 1e-14
    d = diagnostics.charges(phi, P, pl, g, 0.0, V)
    assert abs(d["sigma_top"] - EPS0 * 10.0 * V / L) <= 1e-12 * EPS0 * 10.0 * V / L


def _dense_operator(pl, h, nx, ny, shift):
    """Assemble A + diag(shift) cell by cell from the face conductances (brute force)."""
    eps = pl["eps"]
    nz = eps.size
    n = nx * ny * nz
    M = np.zeros((n, n))
    idx = lambda i, j, k: (k * ny + j) * nx + i  # noqa: E731
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                c = idx(i, j, k)
                M[c, c] += shift[k]
                for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                    nb = idx((i + di) % nx, (j + dj) % ny, k)
                    M[c, c] += eps[k] / h ** 2
                    M[c, nb] -= eps[k] / h ** 2
                for dk in (1, -1):
                    kk = k + dk
                    if 0 <= kk < nz:
                        cond = 2 * eps[k] * eps[kk] / (eps[k] + eps[kk]) / h ** 2
                        M[c, c] += cond
                        M[c, idx(i, j, kk)] -= cond
                    else:
                        M[c, c] += 2 * eps[k] / h ** 2      # electrode at half a cell
    return M


@pytest.mark.parametrize("nx,ny,nz", [(4, 3, 6), (3, 5, 4), (1, 1, 7)])
def test_separable_solver_vs_dense(nx, ny, nz):
    rng = np.random.default_rng(7)
    g = I.make_geometry(nx, ny, [I.de_layer(1, float(e)) for e in rng.uniform(2, 30, nz)])
    pl = oracle.planes(g)
    h = 0.5e-9
    shift = rng.uniform(0, 1e9, nz) * EPS0
    b = rng.standard_normal((nz, ny, nx)) * 1e8
    M = _dense_operator(pl, h, nx, ny, shift)
    x_dense = np.linalg.solve(M, b.ravel()).reshape(b.shape)
    x = poisson.solve_separable(b, pl, h, shift)
    assert np.abs(x - x_dense).max() <= 1e-12 * np.abs(x_dense).max()
    # apply_A agrees with the dense matrix
    y = rng.standard_normal(b.shape)
    assert np.allclose(poisson.apply_A(y, pl, h) + shift[:, None, None] * y,
                       (M @ y.ravel()).reshape(b.shape), rtol=1e-13, atol=1e-13 * np.abs(M).max())


def test_manufactured_solution_second_order():
    """Smooth eps(z) and Phi = sin(2 pi x/L) sin(2 pi y/L) sin(pi z/Lz) + V z/Lz:
    the discrete error falls 4x per halving of h."""
    L, Lz, V = 8e-9, 8e-9, 0.3
    errs = []
    for n in (8, 16, 32):
        h = L / n
        z = (np.arange(n) + 0.5) * h
        x = (np.arange(n) + 0.5) * h
        er = 10.0 + 5.0 * np.sin(np.pi * z / Lz)
        g = I.make_geometry(n, n, [I.de_layer(1, float(e)) for e in er], h=h)
        pl = oracle.planes(g)
        X, Y, Z = np.meshgrid(x, x, z, indexing="ij")
        X, Y, Z = (np.transpose(a, (2, 1, 0)) for a in (X, Y, Z))
        kx, kz = 2 * np.pi / L, np.pi / Lz
        S = np.sin(kx * X) * np.sin(kx * Y)
        phi_ex = S * np.sin(kz * Z) + V * Z / Lz
        eps = EPS0 * (10.0 + 5.0 * np.sin(kz * Z))
        deps = EPS0 * 5.0 * kz * np.cos(kz * Z)
        dphidz = S * kz * np.cos(kz * Z) + V / Lz
        lap = -(2 * kx ** 2 + kz ** 2) * S * np.sin(kz * Z)
        f = -(eps * lap + deps * dphidz)          # f = -div(eps grad phi)
        b = f.copy()
        b[-1] += 2 * pl["eps"][-1] * V / h ** 2
        phi = poisson.solve_separable(b, pl, h)
        errs.append(np.sqrt(np.mean((phi - phi_ex) ** 2)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.85 < r < 2.2 for r in rates), (errs, rates)


# ---------------------------------------------------------------- TDGL ----------------

def landau_root(alpha, beta, gamma, E, lo, hi):
    """Root of alpha P + beta P^3 + gamma P^5 = E on [lo, hi] by bisection."""
    g = lambda P: alpha * P + beta * P ** 3 + gamma * P ** 5 - E  # noqa: E731
    glo = g(lo)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if (g(mid) > 0) == (glo > 0):
            lo, glo = mid, g(mid)
        else:
            hi = mid
    return 0.5 * (lo + hi)


def test_homogeneous_landau_equilibrium():
    """Shorted metal/FE/metal, free P BC, uniform P: Phi stays 0 and P relaxes to
    P0^2 = (-beta + sqrt(beta^2 - 4 alpha gamma)) / (2 gamma)."""
    g = I.make_geometry(4, 4, [I.fe_layer(6)], pbc=I.PBC_FREE)
    pl = oracle.planes(g)
    P = uniform_P(g, 0.1)
    phi = np.zeros(P.shape[1:])
    for _ in range(400):
        P, phi = tdgl.step(P, phi, pl, g, 4e-13, 0.0, 0.0)
    a, b, c = I.HZO["alpha"], I.HZO["beta"], I.HZO["gamma"]
    P0 = math.sqrt((-b + math.sqrt(b * b - 4 * a * c)) / (2 * c))
    assert abs(P0 - 0.1950580) < 1e-6
    assert np.abs(phi).max() < 1e-15
    assert np.abs(P - P0).max() < 1e-12


def test_landau_in_uniform_field():
    """Metal/FE/metal at bias V, uniform P: E = -V/L inside and the steady state
    solves alpha P + beta P^3 + gamma P^5 = E (the sign of the coupling, Eq. TDGL2)."""
    V, n = 0.5, 10
    g = I.make_geometry(3, 3, [I.fe_layer(n)], pbc=I.PBC_FREE)
    pl = oracle.planes(g)
    P = uniform_P(g, 0.19)
    phi = tdgl.solve_poisson(P, np.zeros(P.shape[1:]), pl, g, 0.0, V)
    for _ in range(600):
        P, phi = tdgl.step(P, phi, pl, g, 4e-13, 0.0, V)
    E = -V / (n * g["h"])
    root = landau_root(I.HZO["alpha"], I.HZO["beta"], I.HZO["gamma"], E, 0.13, 0.3)
    assert np.abs(P[0][pl["fe"]] - root).max() < 1e-12
    # the wrong sign of the coupling would give the root for +|E|
    wrong = landau_root(I.HZO["alpha"], I.HZO["beta"], I.HZO["gamma"], -E, 0.13, 0.3)
    assert abs(root - wrong) > 1e-2


def _wall_profile(n, L, P0, w):
    h = L / n
    x = (np.arange(n) + 0.5) * h
    return np.tanh((x - L / 4) / w) * np.tanh((3 * L / 4 - x) / w) * P0, x, h


def test_tanh_domain_wall_truncation_second_order():
    """gamma = 0: P = P0 tanh(x/w), P0 = sqrt(-alpha/beta), w = sqrt(-2 g/alpha) solves
    alpha P + beta P^3 - g P'' = 0; the discrete force on it is O(h^2)."""
    a, b, gg = -2.5e9, 6.0e10, 1e-9
    P0 = math.sqrt(-a / b)
    w = math.sqrt(-2 * gg / a)
    L = 48 * w
    errs = []
    for n in (192, 384, 768):
        h = L / n
        g = I.make_geometry(n, 1, [I.fe_layer(2, g=gg, gamma=0.0)], h=h, pbc=I.PBC_FREE)
        pl = oracle.planes(g)
        prof, x, _ = _wall_profile(n, L, P0, w)
        P = np.zeros((1, 2, 1, n))
        P[0, :, 0, :] = prof
        f = tdgl.force(P, np.zeros(P.shape[1:]), pl, g, 0.0, 0.0)
        # the two-wall product differs from a solution by ~e^-24; measure near walls
        errs.append(np.abs(f).max() / (I.HZO["Gamma"] * abs(a) * P0))
    r1, r2 = math.log2(errs[0] / errs[1]), math.log2(errs[1] / errs[2])
    assert 1.9 < r1 < 2.1 and 1.9 < r2 < 2.1, errs
    # a flipped gradient sign would leave an O(1) force
    assert errs[-1] < 1e-3


def test_tanh_domain_wall_relaxed_equilibrium():
    """Relax the two-wall profile: it stays within O(h^2) of the tanh solution."""
    a, b, gg = -2.5e9, 6.0e10, 1e-9
    P0 = math.sqrt(-a / b)
    w = math.sqrt(-2 * gg / a)
    L, n = 48 * w, 192
    g = I.make_geometry(n, 1, [I.fe_layer(2, g=gg, gamma=0.0)], h=L / n, pbc=I.PBC_FREE)
    pl = oracle.planes(g)
    prof, x, h = _wall_profile(n, L, P0, w)
    P = np.zeros((1, 2, 1, n))
    P[0, :, 0, :] = prof
    phi = np.zeros(P.shape[1:])
    dt = 0.2 * h ** 2 / (I.HZO["Gamma"] * gg)
    for _ in range(3000):
        P, phi = tdgl.step(P, phi, pl, g, dt, 0.0, 0.0)
    err = np.abs(P[0, 0, 0] - prof).max() / P0
    assert err < 5e-3 * (48 / n * 4) ** 2
    assert np.abs(phi).max() < 1e-14


def test_polarization_bc_limits_and_quadratic_exactness():
    h, lam = 0.5e-9, 3e-9
    rng = np.random.default_rng(3)
    P0, P1 = rng.standard_normal(5), rng.standard_normal(5)
    free = tdgl.boundary_face_value(P0, P1, tdgl.PBC_FREE, lam, h)
    assert np.allclose(tdgl.boundary_face_value(P0, P1, tdgl.PBC_LAMBDA, 1e30, h), free, rtol=1e-12)
    assert np.all(tdgl.boundary_face_value(P0, P1, tdgl.PBC_LAMBDA, 0.0, h) == 0.0)
    # quadratic profiles that satisfy each BC exactly: the one-sided stencil is exact
    g = I.make_geometry(1, 1, [I.fe_layer(6)], h=h)
    fe = np.ones(6, dtype=bool)
    s = (np.arange(6) + 0.5) * h          # distance from the bottom face
    c, aa = 0.07, 3e15
    cases = {tdgl.PBC_FREE: c + aa * s ** 2,                      # P'(0) = 0
             tdgl.PBC_ZERO: aa * s * (s - 1e-9),                  # P(0) = 0
             tdgl.PBC_LAMBDA: c + (c / lam) * s + aa * s ** 2}     # lam P'(0) = P(0)
    for pbc, prof in cases.items():
        Pc = prof[:, None, None]
        d2 = tdgl.d2z(Pc, fe, pbc, lam, h)
        assert abs(d2[0, 0, 0] - 2 * aa) <= 1e-9 * 2 * aa, pbc
        assert abs(d2[2, 0, 0] - 2 * aa) <= 1e-9 * 2 * aa
    del g


@pytest.mark.parametrize("order", [1, 2])
def test_integrator_amplification_factor(order):
    """beta = gamma = 0 in a shorted uniform MFM: Phi = 0, dP/dt = -Gamma alpha P, so one
    step multiplies P by 1 - z (order 1) or 1 - z + z^2/2 (Heun, order 2), z = Gamma alpha dt."""
    g = I.make_geometry(2, 2, [I.fe_layer(4, beta=0.0, gamma=0.0)], pbc=I.PBC_FREE)
    pl = oracle.planes(g)
    P = uniform_P(g, 1e-3)
    phi = np.zeros(P.shape[1:])
    dt = 4e-13
    z = I.HZO["Gamma"] * I.HZO["alpha"] * dt
    amp = (1 - z) if order == 1 else (1 - z + 0.5 * z * z)
    for _ in range(5):
        P, phi = tdgl.step(P, phi, pl, g, dt, 0.0, 0.0, order=order)
    assert np.abs(P[0][pl["fe"]] - 1e-3 * amp ** 5).max() <= 1e-14 * 1e-3 * amp ** 5


def _bump_problem(n=16, h=2e-9):
    """Convergence-study set-up of the Numerical Validation section: 32 nm cube,
    bottom 25% undoped Si, 25% dielectric, top 50% FE, lambda = 3 nm, Phi = 0 on both
    faces, Gaussian bump P = 0.002 exp(-(x^2+y^2)/(2 s1^2) - (z - z0)^2/(2 s2^2))."""
    q = n // 4
    layers = [I.sc_layer(q, N_A=0.0, n_i=1e16), I.de_layer(q, I.EPS_SIO2), I.fe_layer(2 * q, g=1e-9)]
    g = I.make_geometry(n, n, layers, h=h, pbc=I.PBC_LAMBDA, lam=3e-9)
    c = (np.arange(n) + 0.5) * h - n * h / 2
    z = (np.arange(n) + 0.5) * h
    Z, Y, X = np.meshgrid(z, c, c, indexing="ij")
    P = 0.002 * np.exp(-(X ** 2 + Y ** 2) / (2 * (5e-9) ** 2) - (Z - 24e-9) ** 2 / (2 * (2e-9) ** 2))
    P[~I.fe_plane_mask(g)] = 0.0
    return g, P[None]


def _paper_convergence_table():
    """The paper's printed convergence table (tests/golden/convergence_table.txt):
    {(test, field): (E_c^m, rate, E_m^f)}."""
    path = os.path.join(os.path.dirname(__file__), "golden", "convergence_table.txt")
    out = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            t, f, ecm, rate, emf = line.split()
            out[(int(t), f)] = (float(ecm), float(rate), float(emf))
    return out


def test_paper_convergence_table_is_consistent():
    """The printed rates are log2 of the printed error ratios (the fixture is read right)."""
    for (t, f), (ecm, rate, emf) in _paper_convergence_table().items():
        assert abs(math.log2(ecm / emf) - rate) < 0.02, (t, f)


@pytest.mark.parametrize("order", [1, 2])
def test_temporal_convergence_rates(order):
    """Convergence table, Tests 1 and 2 (t = 400 fs, dt = 50 / 25 / 12.5 fs): the
    oracle's temporal self-convergence rates of P and Phi match the printed rates
    (1.00 / 1.01 first order, 2.02 / 2.07 second order) within 0.12."""
    table = _paper_convergence_table()
    g, P0 = _bump_problem()
    pl = oracle.planes(g)
    sols = []
    for dt in (50e-15, 25e-15, 12.5e-15):
        steps = int(round(400e-15 / dt))
        sols.append(tdgl.run(P0, pl, g, dt, 0.0, 0.0, steps, order=order))
    for which, field in ((0, "P"), (1, "Phi")):
        e1 = np.sqrt(np.mean((sols[1][which] - sols[0][which]) ** 2))
        e2 = np.sqrt(np.mean((sols[2][which] - sols[1][which]) ** 2))
        rate = math.log2(e1 / e2)
        assert abs(rate - table[(order, field)][1]) < 0.12, (field, rate)


# ---------------------------------------------------------------- carriers -----------

def test_neutral_bulk_at_zero_potential():
    g = I.make_geometry(2, 2, I.mfism_stack(16))
    pl = oracle.planes(g)
    rho, s = carriers.charge(np.zeros((16, 2, 2)), pl)
    assert np.abs(rho).max() <= 1e-15 * Q_E * 1e24
    vt = K_B * 300.0 / Q_E
    assert abs(vt - 0.025852) < 1e-6
    sc = pl["sc"]
    assert np.allclose(s[sc], Q_E * (1e24 + 1e8) / vt, rtol=1e-12)


def test_debye_screening_small_signal():
    """1-D MIS under a tiny bias: in the Si bulk the potential decays by the discrete
    screening factor exp(kappa h), 2 cosh(kappa h) - 2 = h^2 q p0 / (eps V_T), and
    kappa ~ 1/L_D with L_D = sqrt(eps V_T / (q N_A)) = 4.09 nm."""
    h = 0.5e-9
    g = I.make_geometry(1, 1, [I.sc_layer(120), I.de_layer(2, I.EPS_SIO2)], h=h)
    pl = oracle.planes(g)
    P = np.zeros((1, 122, 1, 1))
    b = poisson.rhs(P, pl, h, 0.0, 1e-5)
    phi, _ = carriers.newton_solve(b, np.zeros((122, 1, 1)), pl, h, tol=1e-10)
    col = phi[:, 0, 0]
    vt = K_B * 300.0 / Q_E
    eps = EPS0 * I.EPS_SI
    kappa = math.acosh(1 + h * h * Q_E * 1e24 / (eps * vt) / 2) / h
    ratios = col[100:110] / col[99:109]
    assert np.allclose(ratios, math.exp(kappa * h), rtol=1e-4)
    L_D = math.sqrt(eps * vt / (Q_E * 1e24))
    assert abs(L_D - 4.09e-9) < 0.01e-9
    assert abs(kappa * L_D - 1) < 2e-3


def test_newton_matches_lagged_fixed_point_undoped():
    """Undoped Si (the paper's MFISM): the lagged fixed point of the paper and the
    damped Newton reach the same potential (the nonlinear problem has one solution)."""
    g = I.make_geometry(8, 8, [I.sc_layer(12, N_A=0.0, n_i=1e16), I.de_layer(2), I.fe_layer(8)])
    pl = oracle.planes(g)
    P = I.random_polarization(g, seed=11, amp=0.05)
    b = poisson.rhs(P, pl, g["h"], 0.0, 0.4)
    phi_n, it_n = carriers.newton_solve(b, np.zeros((22, 8, 8)), pl, g["h"])
    phi_f, it_f = carriers.fixed_point_solve(b, np.zeros((22, 8, 8)), pl, g["h"])
    assert np.abs(phi_n - phi_f).max() <= 1e-11 * np.abs(phi_n).max()
    # and Newton from a different start lands on the same point
    phi_n2, _ = carriers.newton_solve(b, np.full((22, 8, 8), 0.3), pl, g["h"])
    assert np.abs(phi_n - phi_n2).max() <= 1e-11 * np.abs(phi_n).max()


def test_newton_doped_residual_and_uniqueness():
    g = I.make_geometry(8, 8, I.mfism_stack(24, n_fe=6, n_ox=2))
    pl = oracle.planes(g)
    P = I.random_polarization(g, seed=12, amp=0.1)
    b = poisson.rhs(P, pl, g["h"], 0.0, 0.8)
    phi_a, _ = carriers.newton_solve(b, np.zeros((24, 8, 8)), pl, g["h"])
    phi_b, _ = carriers.newton_solve(b, np.full((24, 8, 8), -0.2), pl, g["h"])
    assert np.abs(phi_a - phi_b).max() <= 1e-10 * np.abs(phi_a).max()
    rho, _ = carriers.charge(phi_a, pl)
    r = poisson.residual(phi_a, b, pl, g["h"], rho)
    assert np.linalg.norm(r) <= 1e-12 * max(np.linalg.norm(b), np.linalg.norm(rho))


# ---------------------------------------------------------------- 3-component model ---

def test_three_component_reduces_to_uniaxial():
    """With P_x = P_y = 0 the z-force and the bound charge of the 3-component model
    are the uniaxial ones; with laterally uniform P there is no in-plane field, so
    P_x, P_y stay zero and whole runs coincide with the paper's uniaxial model."""
    g1 = I.make_geometry(8, 6, I.mfim_stack(12, n_fe=6))
    g3 = dict(g1, ncomp=3)
    pl = oracle.planes(g1)
    Pz = I.random_polarization(g1, seed=5, amp=0.1)
    phi = np.random.default_rng(6).uniform(-0.3, 0.3, Pz.shape[1:])
    P3 = np.zeros((3,) + Pz.shape[1:])
    P3[2] = Pz[0]
    f1 = tdgl.force(Pz, phi, pl, g1, 0.0, 0.3)
    f3 = tdgl.force(P3, phi, pl, g3, 0.0, 0.3)
    assert np.array_equal(f3[2], f1[0])
    assert np.array_equal(poisson.rhs(P3, pl, g1["h"], 0.0, 0.3), poisson.rhs(Pz, pl, g1["h"], 0.0, 0.3))
    # laterally uniform, z-varying polarization
    col = np.linspace(-0.05, 0.08, 12)[:, None, None] * np.ones((12, 6, 8))
    Pz = col[None] * I.fe_plane_mask(g1)[None, :, None, None]
    P3 = np.zeros((3,) + Pz.shape[1:])
    P3[2] = Pz[0]
    a1 = tdgl.run(Pz, pl, g1, 4e-13, 0.0, 0.3, 3)
    a3 = tdgl.run(P3, pl, g3, 4e-13, 0.0, 0.3, 3)
    assert np.all(np.abs(a3[0][:2]) <= 1e-14)
    assert np.abs(a3[0][2] - a1[0][0]).max() <= 1e-15 * np.abs(a1[0]).max()
    assert np.abs(a3[1] - a1[1]).max() <= 1e-13 * np.abs(a1[1]).max()


def test_in_plane_component_uniform_landau_root():
    """Uniform in-plane P_x in a shorted all-FE stack has no bound charge, so
    Phi = 0 and P_x relaxes to the root of its own Landau polynomial."""
    ax, bx, cx = -1.0e9, 8.0e10, 1.0e11
    g = I.make_geometry(4, 4, [I.fe_layer(6, alpha_xy=ax, beta_xy=bx, gamma_xy=cx)],
                        pbc=I.PBC_FREE, ncomp=3)
    pl = oracle.planes(g)
    P = np.zeros((3, 6, 4, 4))
    P[0] = 0.05
    phi = np.zeros((6, 4, 4))
    for _ in range(800):
        P, phi = tdgl.step(P, phi, pl, g, 4e-13, 0.0, 0.0)
    P0 = math.sqrt((-bx + math.sqrt(bx * bx - 4 * ax * cx)) / (2 * cx))
    assert np.abs(P[0] - P0).max() < 1e-12
    assert np.all(P[1] == 0.0) and np.all(P[2] == 0.0)
    assert np.abs(phi).max() < 1e-15


# ---------------------------------------------------------------- parameters ---------

def test_workload_parameters_match_the_paper_table():
    """The seeded workloads take the paper's parameter table (tests/golden/
    table1_parameters.txt); the gradient coefficient of the workloads is 1e-10
    (the table prints 1e-9; both run), and the FE layer carries g11 = g44."""
    path = os.path.join(os.path.dirname(__file__), "golden", "table1_parameters.txt")
    t = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            t[k] = float(v)
    fe = I.fe_layer(10)
    assert (fe["alpha"], fe["beta"], fe["gamma"]) == (t["alpha"], t["beta"], t["gamma"])
    assert fe["eps_r"] == t["eps_fe"] and fe["Gamma"] == t["Gamma"]
    assert t["g11"] == t["g44"] and fe["g11"] == fe["g44"]
    assert I.fe_layer(10, g=t["g11"])["g11"] == t["g11"]
    assert I.de_layer(4)["eps_r"] == t["eps_sio2"] and I.de_layer(4, 10.0)["eps_r"] == t["eps_al2o3"]
    assert I.sc_layer(4)["eps_r"] == t["eps_sc"]
    assert I.H_DEFAULT == t["h"] and I.LAMBDA_DEFAULT == t["lambda"] and I.DT_DEFAULT == t["dt"]


# ------------------------------------------- in-plane terms of the 3-component model ---
#
# A single lateral Fourier mode of P_x (or P_y) in a shorted all-ferroelectric stack
# has a bound charge -dP_x/dx and a potential known in closed form, both for the
# continuum problem and for the discrete finite-volume operator.  These pin the
# in-plane bound charge of the right-hand side (sign, face average) and the in-plane
# field that drives P_x (sign, face potentials), which laterally uniform cases leave
# untouched.

def _in_plane_stack(nx, ny, nz, h, eps_r=24.0):
    fe = I.fe_layer(nz, g=0.0, alpha=0.0, beta=0.0, gamma=0.0,
                    alpha_xy=0.0, beta_xy=0.0, gamma_xy=0.0, eps_r=eps_r)
    return I.make_geometry(nx, ny, [fe], h=h, pbc=I.PBC_FREE, ncomp=3)


def _mode_P(g, comp, A, m):
    """P_comp = A sin(theta (i + 1/2)) along x (comp 0) or y (comp 1), theta = 2 pi m / n."""
    nz = I.nz_of(g)
    P = np.zeros((3, nz, g["ny"], g["nx"]))
    n = g["nx"] if comp == 0 else g["ny"]
    th = 2.0 * np.pi * m / n
    wave = A * np.sin(th * (np.arange(n) + 0.5))
    P[comp] = wave[None, None, :] if comp == 0 else wave[None, :, None]
    return P, th


@pytest.mark.parametrize("comp,m", [(0, 1), (0, 3), (1, 2)])
def test_in_plane_mode_exact_discrete_potential(comp, m):
    """P_x = A sin(theta (i+1/2)) gives the face-averaged bound charge
    b_i = -A sin(theta) cos(theta (i+1/2))/h, and the discrete operator maps
    cos(theta (i+1/2)) g_k onto itself with lateral eigenvalue eps (2-2cos theta)/h^2.
    The z profile then solves a constant-coefficient recurrence, closed form:
        g_k = G + C cosh(mu (k - (N-1)/2)),  cosh mu = 2 - cos theta,
        G = s/(eps lambda),  s = -A sin(theta)/h,  lambda = (2 - 2cos theta)/h^2,
    with C from the half-cell electrode face (coupling 2 eps/h^2, V = 0)."""
    h, nz, A = 0.5e-9, 8, 0.07
    nx, ny = (16, 2) if comp == 0 else (2, 12)
    g = _in_plane_stack(nx, ny, nz, h)
    pl = oracle.planes(g)
    P, th = _mode_P(g, comp, A, m)
    eps = pl["eps"][0]
    # right-hand side: bound charge of the in-plane mode only
    b = poisson.rhs(P, pl, h, 0.0, 0.0)
    n = nx if comp == 0 else ny
    c = np.cos(th * (np.arange(n) + 0.5))
    lateral = c[None, None, :] if comp == 0 else c[None, :, None]
    s = -A * np.sin(th) / h
    assert np.abs(b - s * lateral * np.ones_like(b)).max() <= 1e-12 * abs(s)
    # potential: exact discrete closed form
    lam = (2.0 - 2.0 * np.cos(th)) / h ** 2
    mu = np.arccosh(2.0 - np.cos(th))
    G = s / (eps * lam)
    mid = 0.5 * (nz - 1)
    c0, c1 = np.cosh(mu * mid), np.cosh(mu * (mid - 1.0))
    C = -(2.0 * eps / h ** 2) * G / (eps * lam * c0 + (2.0 * eps / h ** 2) * c0 + (eps / h ** 2) * (c0 - c1))
    gk = G + C * np.cosh(mu * (np.arange(nz) - mid))
    phi_exact = gk[:, None, None] * lateral
    phi = poisson.solve_linear(P, pl, h, 0.0, 0.0)
    assert np.abs(phi - phi_exact).max() <= 1e-11 * np.abs(phi_exact).max()


@pytest.mark.parametrize("comp", [0, 1])
def test_in_plane_depolarising_force_second_order(comp):
    """Continuum: P_x = A sin(kx) in a shorted film of thickness Lz (eps uniform) gives
    Phi = -(A/(eps k)) cos(kx) u(z), u = 1 - cosh(k(z - Lz/2))/cosh(k Lz/2), so with
    the Landau and gradient terms off the TDGL force on P_x is
        f_x = -Gamma dPhi/dx = -Gamma (A/eps) sin(kx) u(z)
    (a depolarising force against P_x).  The oracle's force converges to it at second
    order; a flipped sign of the bound charge or of the field coupling fails at once."""
    A, L = 0.05, 8e-9
    errs = []
    for n in (32, 64, 128):
        h = L / n
        nz = n // 2
        nx, ny = (n, 2) if comp == 0 else (2, n)
        g = _in_plane_stack(nx, ny, nz, h)
        pl = oracle.planes(g)
        P, _ = _mode_P(g, comp, A, 1)
        phi = poisson.solve_linear(P, pl, h, 0.0, 0.0)
        f = tdgl.force(P, phi, pl, g, 0.0, 0.0)
        eps, Gam = pl["eps"][0], pl["Gamma"][0]
        k = 2.0 * np.pi / L
        xc = (np.arange(n) + 0.5) * h
        zc = (np.arange(nz) + 0.5) * h
        Lz = nz * h
        u = 1.0 - np.cosh(k * (zc - 0.5 * Lz)) / np.cosh(0.5 * k * Lz)
        s = np.sin(k * xc)
        lateral = s[None, None, :] if comp == 0 else s[None, :, None]
        f_exact = -Gam * (A / eps) * u[:, None, None] * lateral
        phi_exact = -(A / (eps * k)) * u[:, None, None] * (np.cos(k * xc)[None, None, :] if comp == 0
                                                          else np.cos(k * xc)[None, :, None])
        errs.append((np.abs(f[comp] - f_exact).max() / np.abs(f_exact).max(),
                     np.abs(phi - phi_exact).max() / np.abs(phi_exact).max()))
        # no field along the uniform lateral direction (P_z is driven by dPhi/dz, which
        # the electrodes make nonzero)
        assert np.all(f[1 - comp] == 0.0)
    # the half-cell electrode closure leaves the coarsest grids slightly pre-asymptotic
    for q in range(2):
        assert errs[0][q] < 0.03
        for a, b in zip(errs, errs[1:]):
            assert 1.75 < math.log2(a[q] / b[q]) < 2.1, errs


@pytest.mark.parametrize("comp", [0, 1])
def test_in_plane_nyquist_mode_zero_displacement(comp):
    """P_x = A (-1)^i: the face averages of P_x vanish, so there is no bound charge and
    Phi = 0 at the cell centres.  With D_x = -eps dPhi/dx + P_x equal to the face flux
    (zero) in every half-cell, the field inside each cell is E_x = -P_x/eps, and the
    TDGL force (Landau and gradient off) is f_x = Gamma E_x = -Gamma P_x/eps."""
    h, nz, A = 0.5e-9, 6, 0.03
    nx, ny = (8, 2) if comp == 0 else (2, 10)
    g = _in_plane_stack(nx, ny, nz, h)
    pl = oracle.planes(g)
    P, _ = _mode_P(g, comp, A, (nx if comp == 0 else ny) // 2)
    # sin(pi (i + 1/2)) = (-1)^i
    alt = (-1.0) ** np.arange(nx if comp == 0 else ny)
    assert np.abs(P[comp] - A * (alt[None, None, :] if comp == 0 else alt[None, :, None])).max() < 1e-15
    phi = poisson.solve_linear(P, pl, h, 0.0, 0.0)
    assert np.abs(phi).max() <= 1e-25
    f = tdgl.force(P, phi, pl, g, 0.0, 0.0)
    eps, Gam = pl["eps"][0], pl["Gamma"][0]
    assert np.abs(f[comp] + Gam * P[comp] / eps).max() <= 1e-13 * Gam * A / eps


# ------------------------------------------- Fermi-Dirac carriers (the paper's model) ---

def _fd_quad(eta, order=0.5):
    """(1/Gamma(order+1)) int_0^inf x^order/(1+e^(x-eta)) dx by adaptive quadrature (order
    1/2: F_1/2 normalised to e^eta for eta -> -inf; order -1/2: its exact derivative)."""
    from scipy import integrate, special
    f = lambda x: x ** order / (1.0 + math.exp(x - eta)) if x - eta < 700 else 0.0  # noqa: E731
    v, _ = integrate.quad(f, 0.0, max(eta, 0.0) + 60.0, limit=400, epsabs=0.0, epsrel=1e-12)
    return v / special.gamma(order + 1.0)


def test_fd_half_approximation_against_quadrature():
    """The Fermi-Dirac integral of order 1/2 of the paper's carrier model, by the
    approximation the paper cites, agrees with the integral itself (quadrature of
    Eq. ne's integrand) within the approximation's accuracy (0.4%), and has the
    right limits: e^eta (non-degenerate, Boltzmann) and (4/(3 sqrt pi)) eta^(3/2)
    (fully degenerate)."""
    etas = np.linspace(-20.0, 40.0, 241)
    rel = [abs(float(carriers.fd_half(e)) / _fd_quad(e) - 1.0) for e in etas]
    assert max(rel) <= 4e-3, max(rel)
    assert abs(float(carriers.fd_half(-30.0)) / math.exp(-30.0) - 1.0) < 1e-9
    big = 1e4
    assert abs(float(carriers.fd_half(big)) / (4.0 / (3.0 * math.sqrt(math.pi)) * big ** 1.5) - 1.0) < 1e-6


def test_fd_half_derivative():
    """The Newton Jacobian uses the derivative of the approximation: it matches a
    central difference of the approximation, and the exact derivative of F_1/2
    (which is F_-1/2) within a few per cent."""
    for e in (-15.0, -3.0, -1.0, 0.0, 0.7, 2.5, 8.0, 25.0):
        d = float(carriers.fd_half_deriv(e))
        h = 1e-5 * max(1.0, abs(e))
        fd = (float(carriers.fd_half(e + h)) - float(carriers.fd_half(e - h))) / (2 * h)
        assert abs(d / fd - 1.0) < 1e-6, (e, d, fd)
        assert abs(d / _fd_quad(e, -0.5) - 1.0) < 0.03, (e, d)


def test_effective_density_of_states_silicon():
    """N = 2 (2 pi m* k_B T / h^2)^(3/2) with the paper's effective masses (Table 1:
    1.08 and 0.81 m_e) gives the textbook 300 K silicon values 2.8e19 and 1.83e19 cm^-3."""
    assert abs(carriers.effective_dos(1.08, 300.0) / 2.8e25 - 1.0) < 0.01
    assert abs(carriers.effective_dos(0.81, 300.0) / 1.83e25 - 1.0) < 0.01
    # T^(3/2) and m^(3/2)
    assert abs(carriers.effective_dos(1.08, 600.0) / carriers.effective_dos(1.08, 300.0) - 2 ** 1.5) < 1e-12


def _fd_stack(N_A=0.0, N_D=0.0, nsc=12, nx=4, ny=4):
    return I.make_geometry(nx, ny, [I.sc_layer(nsc, N_A=N_A, N_D=N_D, stats=I.STATS_FERMI_DIRAC),
                                    I.de_layer(2), I.fe_layer(6)], pbc=I.PBC_FREE)


@pytest.mark.parametrize("N_A,N_D", [(0.0, 0.0), (1e24, 0.0), (0.0, 3e23), (1e26, 0.0)])
def test_fd_bulk_neutral_at_zero_potential(N_A, N_D):
    """The band edges are placed so that the semiconductor bulk is neutral at Phi = 0
    (ohmic contact at V0 = 0), for undoped, p-, n- and degenerately doped Si; the
    carrier densities obey the mass-action law n p = N_c N_v F(eta_e)F(eta_p) and, for
    undoped Si, n = p = n_i = sqrt(N_c N_v) exp(-E_g/2k_BT) to the Boltzmann limit."""
    g = _fd_stack(N_A, N_D)
    pl = oracle.planes(g)
    phi = np.zeros((I.nz_of(g), 4, 4))
    rho, s = carriers.charge(phi, pl)
    scale = Q_E * max(N_A, N_D, 1e16)
    assert np.abs(rho).max() <= 1e-12 * scale
    assert np.all(s[pl["sc"]] > 0.0)
    if N_A == 0.0 and N_D == 0.0:
        Nc, Nv = carriers.effective_dos(1.08, 300.0), carriers.effective_dos(0.81, 300.0)
        ee, ep = carriers.fd_reference(Nc, Nv, 1.12, 300.0, 0.0, 0.0)
        n_i = math.sqrt(Nc * Nv) * math.exp(-1.12 * Q_E / (2 * K_B * 300.0))
        assert abs(Nc * float(carriers.fd_half(ee)) / n_i - 1.0) < 1e-6
        assert abs(Nv * float(carriers.fd_half(ep)) / n_i - 1.0) < 1e-6


def test_fd_reduces_to_boltzmann_when_non_degenerate():
    """Undoped Si at moderate potentials is non-degenerate, so the Fermi-Dirac charge
    and its derivative equal the Maxwell-Boltzmann ones (Eq. MaxBolt_ne_np) with the
    same intrinsic density, to the size of e^eta."""
    g_fd = _fd_stack()
    pl_fd = oracle.planes(g_fd)
    Nc, Nv = carriers.effective_dos(1.08, 300.0), carriers.effective_dos(0.81, 300.0)
    n_i = math.sqrt(Nc * Nv) * math.exp(-1.12 * Q_E / (2 * K_B * 300.0))
    g_mb = I.make_geometry(4, 4, [I.sc_layer(12, N_A=0.0, n_i=n_i), I.de_layer(2), I.fe_layer(6)],
                           pbc=I.PBC_FREE)
    pl_mb = oracle.planes(g_mb)
    phi = np.random.default_rng(3).uniform(-0.25, 0.25, (20, 4, 4))
    r_fd, s_fd = carriers.charge(phi, pl_fd)
    r_mb, s_mb = carriers.charge(phi, pl_mb)
    sc = pl_fd["sc"]
    assert np.abs(r_fd[sc] - r_mb[sc]).max() <= 1e-4 * np.abs(r_mb[sc]).max()
    assert np.abs(s_fd[sc] / s_mb[sc] - 1.0).max() <= 1e-4


def test_fd_degenerate_density():
    """Deep in the conduction band the electron density is the degenerate limit
    N_c (4/(3 sqrt pi)) eta^(3/2), far below the Boltzmann exponential."""
    g = _fd_stack(N_D=1e24)
    pl = oracle.planes(g)
    Nc, Nv = carriers.effective_dos(1.08, 300.0), carriers.effective_dos(0.81, 300.0)
    ee, _ = carriers.fd_reference(Nc, Nv, 1.12, 300.0, 0.0, 1e24)
    vt = K_B * 300.0 / Q_E
    phi = np.zeros((20, 4, 4))
    phi[:12] = 3.0                                      # eta_e ~ 110
    rho, _ = carriers.charge(phi, pl)
    eta = ee + 3.0 / vt
    n_deg = Nc * 4.0 / (3.0 * math.sqrt(math.pi)) * eta ** 1.5
    n = -(rho[0, 0, 0] / Q_E - 1e24)                    # p is negligible here
    assert abs(n / n_deg - 1.0) < 1e-3
    assert n < 1e-30 * Nc * math.exp(eta)


def test_fd_newton_matches_lagged_fixed_point_undoped():
    """The paper's MFISM with undoped Si and Fermi-Dirac carriers: the damped Newton
    solve and the paper's lagged fixed point (Methods, "Numerical Approach") reach the
    same potential (the problem has one solution)."""
    g = I.make_geometry(8, 6, [I.sc_layer(10, N_A=0.0, stats=I.STATS_FERMI_DIRAC), I.de_layer(4),
                               I.fe_layer(8)], pbc=I.PBC_LAMBDA)
    pl = oracle.planes(g)
    P = I.random_polarization(g, seed=4, amp=0.15)
    b = poisson.rhs(P, pl, g["h"], 0.0, 0.8)
    phi_n, _ = carriers.newton_solve(b, np.zeros(P.shape[1:]), pl, g["h"], tol=1e-14)
    phi_f, _ = carriers.fixed_point_solve(b, np.zeros(P.shape[1:]), pl, g["h"], tol=1e-15)
    assert np.abs(phi_n - phi_f).max() <= 1e-12 * np.abs(phi_f).max()
    rho, _ = carriers.charge(phi_n, pl)
    assert np.abs(rho).max() > 0.0


# ------------------------------------------------------------ Q-V sweep protocol -------

def test_triangle_wave_protocol():
    """0 -> +Vmax -> 0 -> -Vmax -> 0 in equal steps, repeated per sweep."""
    v = I.triangle_wave(2.0, 4, sweeps=2)
    assert len(v) == 32
    assert v[:4] == [0.5, 1.0, 1.5, 2.0] and v[4:8] == [1.5, 1.0, 0.5, 0.0]
    assert v[8:12] == [-0.5, -1.0, -1.5, -2.0] and v[12:16] == [-1.5, -1.0, -0.5, 0.0]
    assert v[16:] == v[:16]


def test_qv_sweep_linear_capacitor():
    """With the ferroelectric frozen at P = 0 (Gamma = 0) the stack is two dielectrics
    in series: every recorded point has Q = V_app / (t_de/eps_de + t_fe/eps_fe) and
    V_fe = Q t_fe/eps_fe, whatever the path, so the protocol's bookkeeping (bias order,
    signs, which state is recorded) is pinned by the series-capacitor closed form."""
    h = 0.5e-9
    g = I.make_geometry(4, 4, [I.de_layer(8, 10.0), I.fe_layer(10, Gamma=0.0)], h=h, pbc=I.PBC_FREE)
    pl = oracle.planes(g)
    P0 = np.zeros((1, 18, 4, 4))
    v = I.triangle_wave(3.0, 3)
    rec, P, _ = diagnostics.qv_sweep(P0, np.zeros((18, 4, 4)), pl, g, 4e-13, v, 2)
    t_de, t_fe = 8 * h, 10 * h
    c_series = 1.0 / (t_de / (10.0 * EPS0) + t_fe / (24.0 * EPS0))
    for vq, r in zip(v, rec):
        assert abs(r["Q_int"] - c_series * vq) <= 1e-12 * c_series * 3.0
        assert abs(r["V_fe"] - r["Q_int"] * t_fe / (24.0 * EPS0)) <= 1e-12 * 3.0
    assert np.all(P == 0.0)

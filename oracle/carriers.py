"""Semiconductor charge and the nonlinear Poisson solve (oracle; test infrastructure).

Charge density (Eq. rho): rho = e [n_p - n_e + N_d - N_a] in semiconductor cells.
Carrier densities, per layer (its "stats" field):
  * Maxwell-Boltzmann limit of the Fermi-Dirac integrals (Eq. MaxBolt_ne_np),
    written with the intrinsic density n_i and the potential referenced so that
    the bulk is neutral at Phi = 0 (an ohmic contact at V0 = 0):
        n_e = n0 exp(Phi/V_T),  n_p = p0 exp(-Phi/V_T),  V_T = k_B T / e,
        p-type (N = N_d - N_a <= 0): p0 = -N/2 + sqrt(N^2/4 + n_i^2), n0 = n_i^2/p0
        n-type (N > 0):              n0 =  N/2 + sqrt(N^2/4 + n_i^2), p0 = n_i^2/n0
    so that n0 p0 = n_i^2 and rho(0) = 0.
  * Fermi-Dirac statistics, the paper's model (Eqs. FD, density_state, ne, np):
    with the density of states of a parabolic band the electron integral is
        n_e = N_c F_1/2(eta_e),  eta_e = (e Phi - E_c)/(k_B T),
        N_c = 2 (2 pi m_e* k_B T / h^2)^(3/2)   (effective density of states),
    and the hole integral n_p = N_v F_1/2(eta_p), eta_p = (E_v - e Phi)/(k_B T),
    where F_1/2(eta) = (2/sqrt(pi)) int_0^inf sqrt(x)/(1 + e^(x - eta)) dx is
    evaluated, as in the paper (Methods, "Numerical Approach"), by the
    approximation of Bednarczyk & Bednarczyk (Phys. Lett. A 64, 409 (1978)):
        F_1/2(eta) = 1/(e^(-eta) + xi(eta)),   xi = (3 sqrt(pi)/4) v^(-3/8),
        v = eta^4 + 50 + 33.6 eta [1 - 0.68 exp(-0.17 (eta + 1)^2)].
    Reading (the paper gives no band edges): the band gap E_g is a layer
    parameter, and E_c, E_v (measured from the contact's Fermi level, Phi = 0)
    are placed so that the bulk is neutral at Phi = 0, as for the Boltzmann
    reading: N_v F(eta_p0) - N_c F(eta_e0) + N_d - N_a = 0, eta_e0 + eta_p0 =
    -E_g/(k_B T), solved by bisection.  Then eta_e = eta_e0 + Phi/V_T and
    eta_p = eta_p0 - Phi/V_T.

Nonlinear problem A Phi = b + rho(Phi).  -rho'(Phi) = e (n_e + n_p)/V_T > 0 and A
is SPD, so the problem is strictly monotone and has one solution; any
convergent iteration reaches it.  The paper iterates a lagged fixed point
(Methods, "Numerical Approach": solve with rho(Phi^k) on the right, stop when
the mean |change| < tol).  The oracle solves by damped Newton (same solution),
each Newton system (A + diag(s)) delta = F solved by preconditioned conjugate
gradients with the exact separable solver of A + (plane mean of s) as
preconditioner; the lagged fixed point is kept for comparison.
"""
import numpy as np

from .stack import Q_E, K_B
from . import poisson


def equilibrium_densities(N_A, N_D, n_i):
    """(n0, p0) per plane: neutral, mass-action carrier densities at Phi = 0."""
    N = N_D - N_A
    root = np.sqrt(0.25 * N * N + n_i * n_i)
    n0 = np.zeros_like(N)
    p0 = np.zeros_like(N)
    ptype = N <= 0
    p0[ptype] = -0.5 * N[ptype] + root[ptype]
    with np.errstate(divide="ignore", invalid="ignore"):
        n0[ptype] = np.where(p0[ptype] > 0, n_i[ptype] ** 2 / p0[ptype], 0.0)
    ntype = ~ptype
    n0[ntype] = 0.5 * N[ntype] + root[ntype]
    p0[ntype] = n_i[ntype] ** 2 / n0[ntype]
    return n0, p0


H_PLANCK = 6.62607015e-34     # J s (exact SI)
M_E = 9.1093837015e-31        # kg (CODATA 2018)
STATS_BOLTZMANN, STATS_FERMI_DIRAC = 0, 1


def fd_half(eta):
    """F_1/2(eta) by the Bednarczyk approximation (see the module docstring)."""
    eta = np.asarray(eta, dtype=np.float64)
    w = 1.0 - 0.68 * np.exp(-0.17 * (eta + 1.0) ** 2)
    v = eta ** 4 + 50.0 + 33.6 * eta * w
    xi = 0.75 * np.sqrt(np.pi) * v ** (-0.375)
    with np.errstate(over="ignore"):
        return 1.0 / (np.exp(-eta) + xi)


def fd_half_deriv(eta):
    """d F_1/2 / d eta of the same approximation (the Newton Jacobian's carrier term)."""
    eta = np.asarray(eta, dtype=np.float64)
    g = np.exp(-0.17 * (eta + 1.0) ** 2)
    w = 1.0 - 0.68 * g
    v = eta ** 4 + 50.0 + 33.6 * eta * w
    dv = 4.0 * eta ** 3 + 33.6 * w + 33.6 * eta * 0.68 * g * 0.34 * (eta + 1.0)
    xi = 0.75 * np.sqrt(np.pi) * v ** (-0.375)
    dxi = -0.375 * xi * dv / v
    with np.errstate(over="ignore", invalid="ignore"):
        em = np.exp(-eta)
        d = (em - dxi) / (em + xi) ** 2
    return np.where(np.isfinite(em), d, 0.0)


def effective_dos(m_rel, T):
    """N = 2 (2 pi m* k_B T / h^2)^(3/2), m* = m_rel m_e (effective density of states, m^-3)."""
    return 2.0 * (2.0 * np.pi * m_rel * M_E * K_B * T / H_PLANCK ** 2) ** 1.5


def fd_reference(Nc, Nv, Eg_eV, T, N_A, N_D):
    """(eta_e0, eta_p0): reduced band-edge distances at Phi = 0 that make the bulk neutral."""
    gap = Eg_eV * Q_E / (K_B * T)
    net = lambda ee: Nv * fd_half(-gap - ee) - Nc * fd_half(ee) + N_D - N_A  # noqa: E731
    lo, hi = -gap - 60.0, 60.0            # net(lo) > 0 > net(hi): decreasing in eta_e0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if net(mid) > 0.0:
            lo = mid
        else:
            hi = mid
    ee = 0.5 * (lo + hi)
    return ee, -gap - ee


def charge(phi, pl):
    """(rho, s) on every cell: rho = e(p - n + N_D - N_A), s = -d rho/d Phi."""
    sc = pl["sc"]
    rho = np.zeros_like(phi)
    s = np.zeros_like(phi)
    if not sc.any():
        return rho, s
    n0, p0 = equilibrium_densities(pl["N_A"], pl["N_D"], pl["n_i"])
    stats = pl.get("stats", np.zeros(len(sc), dtype=np.int64))
    for k in np.nonzero(sc)[0]:
        vt = K_B * pl["T"][k] / Q_E
        if stats[k] == STATS_FERMI_DIRAC:
            Nc = effective_dos(pl["m_e"][k], pl["T"][k])
            Nv = effective_dos(pl["m_p"][k], pl["T"][k])
            ee, ep = fd_reference(Nc, Nv, pl["E_g"][k], pl["T"][k], pl["N_A"][k], pl["N_D"][k])
            u = phi[k] / vt
            n = Nc * fd_half(ee + u)
            p = Nv * fd_half(ep - u)
            dn = Nc * fd_half_deriv(ee + u) / vt          # d n / d Phi
            dp = -Nv * fd_half_deriv(ep - u) / vt         # d p / d Phi
            rho[k] = Q_E * (p - n + pl["N_D"][k] - pl["N_A"][k])
            s[k] = -Q_E * (dp - dn)
        else:
            n = n0[k] * np.exp(phi[k] / vt)
            p = p0[k] * np.exp(-phi[k] / vt)
            rho[k] = Q_E * (p - n + pl["N_D"][k] - pl["N_A"][k])
            s[k] = Q_E * (n + p) / vt
    return rho, s


def _pcg(apply_M, rhs_, precond, tol, maxit=500):
    x = np.zeros_like(rhs_)
    r = rhs_.copy()
    z = precond(r)
    p = z.copy()
    rz = np.vdot(r, z)
    nrm0 = np.linalg.norm(rhs_)
    if nrm0 == 0.0:
        return x
    for _ in range(maxit):
        Ap = apply_M(p)
        alpha = rz / np.vdot(p, Ap)
        x += alpha * p
        r -= alpha * Ap
        if np.linalg.norm(r) <= tol * nrm0:
            break
        z = precond(r)
        rz_new = np.vdot(r, z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x


def newton_solve(b, phi0, pl, h, tol=1e-13, max_newton=60):
    """Solve A Phi = b + rho(Phi) by damped Newton.  Returns (Phi, iterations).

    Stops when ||b + rho - A Phi|| <= tol * max(||b||, ||rho||).
    """
    phi = phi0.copy()
    for it in range(max_newton):
        rho, s = charge(phi, pl)
        F = poisson.residual(phi, b, pl, h, rho)
        nF = np.linalg.norm(F)
        scale = max(np.linalg.norm(b), np.linalg.norm(rho))
        if nF <= tol * scale or nF == 0.0:
            return phi, it
        shift = s.mean(axis=(1, 2))
        delta = _pcg(lambda v: poisson.apply_A(v, pl, h) + s * v, F,
                     lambda v: poisson.solve_separable(v, pl, h, shift), tol=1e-3 * tol)
        t = 1.0
        while True:          # backtracking on the residual norm
            trial = phi + t * delta
            rho_t, _ = charge(trial, pl)
            if np.linalg.norm(poisson.residual(trial, b, pl, h, rho_t)) < nF or t < 1e-6:
                break
            t *= 0.5
        phi = trial
    raise RuntimeError("oracle Newton did not converge")


def fixed_point_solve(b, phi0, pl, h, tol=1e-13, max_it=500):
    """The paper's lagged iteration A Phi^(k+1) = b + rho(Phi^(k)); converges only
    while the carrier response is weak (e.g. undoped Si).  Returns (Phi, iterations)."""
    phi = phi0.copy()
    for it in range(max_it):
        rho, _ = charge(phi, pl)
        new = poisson.solve_separable(b + rho, pl, h)
        if np.max(np.abs(new - phi)) <= tol * max(1.0, np.max(np.abs(new))):
            return new, it + 1
        phi = new
    raise RuntimeError("lagged fixed point did not converge")

"""Semiconductor charge and the nonlinear Poisson solve (oracle; test infrastructure).

Charge density (Eq. rho): rho = e [n_p - n_e + N_d - N_a] in semiconductor cells.
Carrier densities: Maxwell-Boltzmann limit of the Fermi-Dirac integrals
(Eq. MaxBolt_ne_np), written with the intrinsic density n_i and the potential
referenced so that the bulk is neutral at Phi = 0 (an ohmic contact at V0 = 0):
    n_e = n0 exp(Phi/V_T),  n_p = p0 exp(-Phi/V_T),  V_T = k_B T / e,
    p-type (N = N_d - N_a <= 0): p0 = -N/2 + sqrt(N^2/4 + n_i^2), n0 = n_i^2/p0
    n-type (N > 0):              n0 =  N/2 + sqrt(N^2/4 + n_i^2), p0 = n_i^2/n0
so that n0 p0 = n_i^2 and rho(0) = 0.

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


def charge(phi, pl):
    """(rho, s) on every cell: rho = e(p - n + N_D - N_A), s = -d rho/d Phi = e(n+p)/V_T."""
    sc = pl["sc"]
    rho = np.zeros_like(phi)
    s = np.zeros_like(phi)
    if not sc.any():
        return rho, s
    n0, p0 = equilibrium_densities(pl["N_A"], pl["N_D"], pl["n_i"])
    for k in np.nonzero(sc)[0]:
        vt = K_B * pl["T"][k] / Q_E
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

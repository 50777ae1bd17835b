"""TDGL polarization dynamics and the coupled time step (oracle; test infrastructure).

Eq. TDGL2 (uniaxial, P = P_z):
    -(1/Gamma) dP/dt = alpha P + beta P^3 + gamma P^5
                       - g44 d2P/dx2 - g44 d2P/dy2 - g11 d2P/dz2 + dPhi/dz.
The electrostatic term enters as +dPhi/dz = -E_z (Eq. TDGL2; this fixes the
sign of the coupling that Eq. elec leaves ambiguous).

Readings (the paper states the boundary conditions but not their stencils):
  * x, y: periodic three-point second differences (Methods, P boundary conditions).
  * z, inside the ferroelectric: three-point second difference.  At a cell next
    to a ferroelectric boundary face (electrode or dielectric), the boundary
    condition gives a face value P_b, and the second derivative uses the
    second-order one-sided stencil through (face, P_0, P_1) at distances
    (0, h/2, 3h/2):
        dP/dn_in(face) = (9 P_0 - P_1 - 8 P_b) / (3h)
        d2P/dz2(cell)  = 4 (P_1 - 3 P_0 + 2 P_b) / (3 h^2)
    with P_b from Eq. Pbc written as lambda dP/dn_in = P at both faces (the
    polarization is reduced at the surface for lambda > 0):
        lambda BC: P_b = lambda (9 P_0 - P_1) / (3h + 8 lambda)
        free  (Eq. PbcFree, lambda -> inf): P_b = (9 P_0 - P_1) / 8
        zero  (Eq. PbcDir, lambda = 0):     P_b = 0
  * dPhi/dz in a cell is the difference of its two face potentials over h;
    face potentials follow from the same flux continuity as the Poisson
    fluxes: electrode face = V; interior face
        Phi_f = (eps_L Phi_L + eps_R Phi_R)/(eps_L + eps_R)
                - (h/2)(P_R - P_L)/(eps_L + eps_R).
  * 3-component model (P_x, P_y, P_z): each component relaxes in its own
    Landau polynomial (alpha_xy... for x and y), the same gradient operator and
    P boundary conditions, and couples to dPhi/dx_i (in-plane face potentials
    with equal eps on both sides).  The paper treats only the uniaxial case and
    names the in-plane components as future work; this is an extension.
"""
import numpy as np

from . import poisson
from . import carriers

PBC_FREE, PBC_ZERO, PBC_LAMBDA = 0, 1, 2


def boundary_face_value(P0, P1, pbc, lam, h):
    """P on a ferroelectric boundary face from the P boundary condition."""
    if pbc == PBC_FREE:
        return (9.0 * P0 - P1) / 8.0
    if pbc == PBC_ZERO:
        return np.zeros_like(P0)
    return lam * (9.0 * P0 - P1) / (3.0 * h + 8.0 * lam)


def d2z(Pc, fe, pbc, lam, h):
    """Second z derivative of one component on ferroelectric planes (0 elsewhere)."""
    nz = Pc.shape[0]
    out = np.zeros_like(Pc)
    for k in range(nz):
        if not fe[k]:
            continue
        below = k > 0 and fe[k - 1]
        above = k < nz - 1 and fe[k + 1]
        if below and above:
            out[k] = (Pc[k + 1] - 2.0 * Pc[k] + Pc[k - 1]) / h ** 2
        elif above:
            Pb = boundary_face_value(Pc[k], Pc[k + 1], pbc, lam, h)
            out[k] = 4.0 * (Pc[k + 1] - 3.0 * Pc[k] + 2.0 * Pb) / (3.0 * h ** 2)
        elif below:
            Pb = boundary_face_value(Pc[k], Pc[k - 1], pbc, lam, h)
            out[k] = 4.0 * (Pc[k - 1] - 3.0 * Pc[k] + 2.0 * Pb) / (3.0 * h ** 2)
        else:
            raise ValueError("a ferroelectric layer must be at least two cells thick")
    return out


def lap_xy(Pc, h):
    return (np.roll(Pc, 1, 2) + np.roll(Pc, -1, 2) + np.roll(Pc, 1, 1) + np.roll(Pc, -1, 1)
            - 4.0 * Pc) / h ** 2


def z_face_potential(phi, Pz, eps, h, v_bottom, v_top):
    """Potential on the Nz+1 z faces of every column."""
    nz = phi.shape[0]
    out = np.empty((nz + 1,) + phi.shape[1:])
    out[0] = v_bottom
    out[nz] = v_top
    eL = eps[:-1, None, None]
    eR = eps[1:, None, None]
    out[1:nz] = ((eL * phi[:-1] + eR * phi[1:]) / (eL + eR)
                 - 0.5 * h * (Pz[1:] - Pz[:-1]) / (eL + eR))
    return out


def dphi_dz(phi, P, pl, h, v_bottom, v_top):
    pf = z_face_potential(phi, P[-1], pl["eps"], h, v_bottom, v_top)
    return (pf[1:] - pf[:-1]) / h


def dphi_dlateral(phi, Pc, eps, h, axis):
    """dPhi/dx (axis 2) or dPhi/dy (axis 1) from in-plane face potentials."""
    e = eps[:, None, None]
    up = 0.5 * (phi + np.roll(phi, -1, axis)) - 0.25 * h * (np.roll(Pc, -1, axis) - Pc) / e
    dn = 0.5 * (np.roll(phi, 1, axis) + phi) - 0.25 * h * (Pc - np.roll(Pc, 1, axis)) / e
    return (up - dn) / h


def force(P, phi, pl, geom, v_bottom, v_top):
    """f(P, Phi) = dP/dt of Eq. TDGL2 on ferroelectric cells (zero elsewhere)."""
    h = geom["h"]
    fe = pl["fe"]
    ncomp = P.shape[0]
    f = np.zeros_like(P)
    s = lambda a: a[:, None, None]  # noqa: E731  (per-plane broadcast)
    for c in range(ncomp):
        Pc = P[c]
        is_z = c == ncomp - 1
        a = pl["alpha"] if is_z else pl["alpha_xy"]
        b = pl["beta"] if is_z else pl["beta_xy"]
        g = pl["gamma"] if is_z else pl["gamma_xy"]
        if is_z:
            dphi = dphi_dz(phi, P, pl, h, v_bottom, v_top)
        else:
            dphi = dphi_dlateral(phi, Pc, pl["eps"], h, axis=2 if c == 0 else 1)
        dF = (s(a) * Pc + s(b) * Pc ** 3 + s(g) * Pc ** 5
              - s(pl["g44"]) * lap_xy(Pc, h)
              - s(pl["g11"]) * d2z(Pc, fe, geom["pbc"], geom["lam"], h)
              + dphi)
        fc = -s(pl["Gamma"]) * dF
        fc[~fe] = 0.0
        f[c] = fc
    return f


def solve_poisson(P, phi_guess, pl, geom, v_bottom, v_top, tol=1e-13):
    """Phi for given P: exact separable solve, or damped Newton with semiconductor."""
    if not pl["sc"].any():
        return poisson.solve_linear(P, pl, geom["h"], v_bottom, v_top)
    b = poisson.rhs(P, pl, geom["h"], v_bottom, v_top)
    return carriers.newton_solve(b, phi_guess, pl, geom["h"], tol=tol)[0]


def step(P, phi, pl, geom, dt, v_bottom, v_top, order=1):
    """One time step (Methods, predictor Steps 1a/1b, corrector Steps 2a/2b)."""
    f0 = force(P, phi, pl, geom, v_bottom, v_top)
    P_star = P + dt * f0                                        # Step 1a
    phi_star = solve_poisson(P_star, phi, pl, geom, v_bottom, v_top)   # Step 1b
    if order == 1:
        return P_star, phi_star
    f1 = force(P_star, phi_star, pl, geom, v_bottom, v_top)
    P_new = P + 0.5 * dt * (f0 + f1)                            # Step 2a
    phi_new = solve_poisson(P_new, phi_star, pl, geom, v_bottom, v_top)  # Step 2b
    return P_new, phi_new


def run(P0, pl, geom, dt, v_bottom, v_top, steps, order=1, phi0=None):
    """Step 0 (initial solve, Methods INITIALIZATION) followed by `steps` time steps."""
    phi = solve_poisson(P0, np.zeros(P0.shape[1:]) if phi0 is None else phi0,
                        pl, geom, v_bottom, v_top)
    P = P0.copy()
    for _ in range(steps):
        P, phi = step(P, phi, pl, geom, dt, v_bottom, v_top, order)
    return P, phi

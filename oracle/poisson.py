"""Variable-permittivity Poisson problem, finite-volume form (oracle; test infrastructure).

Equation (Eq. Poisson and the overview's Poisson equation):
    div(eps grad Phi) = div P - rho,
i.e. div D = rho with D = -eps grad Phi + P.  Boundary conditions (Methods,
"Electrical boundary conditions"): periodic in x and y, Phi = V0 on the bottom
face z = 0 and Phi = V1 on the top face z = Nz h.

Discretisation (a reading; the paper only states second order within each
material).  Cell-centred unknowns on a uniform grid of spacing h.  For every
cell the outward face fluxes F (normal component of D) satisfy
    sum_faces F_out / h = rho_cell.
  * x/y faces (same material on both sides):  F = -eps_k (Phi_R - Phi_L)/h
    (+ the face average of P_x / P_y in the 3-component model).
  * interior z face between cells L (below) and R (above): the flux is taken
    continuous through a face potential, with eps and P uniform in each
    half-cell, which gives
        F = -eps_h (Phi_R - Phi_L)/h + P_f,
        eps_h = 2 eps_L eps_R / (eps_L + eps_R),
        P_f   = (eps_R P_L + eps_L P_R) / (eps_L + eps_R).
    This reproduces the piecewise-linear potential of a layered stack exactly.
  * electrode faces (half-cell distance to the Dirichlet value):
        top:    F = -eps_top (V1 - Phi_top)/(h/2) + P_top
        bottom: F = -eps_bot (Phi_bot - V0)/(h/2) + P_bot.
Written as A Phi = b + rho with A the symmetric positive-definite operator
    (A Phi)_c = sum_faces c_f (Phi_c - Phi_nb)
and b = -(sum of outward P_f)/h + Dirichlet lift 2 eps V/h^2 on boundary planes.
"""
import numpy as np


def face_eps(eps):
    """Harmonic-mean permittivity of the Nz-1 interior z faces (k+1/2, k = 0..Nz-2)."""
    return 2.0 * eps[:-1] * eps[1:] / (eps[:-1] + eps[1:])


def face_polarization(Pz, eps):
    """P_f on all Nz+1 z faces of every column; Pz has shape (Nz, Ny, Nx).

    Electrode faces take the adjacent cell's P; interior faces the eps-weighted
    combination of the two half-cells (flux continuity).
    """
    nz = Pz.shape[0]
    Pf = np.empty((nz + 1,) + Pz.shape[1:])
    Pf[0] = Pz[0]
    Pf[nz] = Pz[nz - 1]
    eL = eps[:-1, None, None]
    eR = eps[1:, None, None]
    Pf[1:nz] = (eR * Pz[:-1] + eL * Pz[1:]) / (eL + eR)
    return Pf


def rhs(P, pl, h, v_bottom, v_top):
    """Right-hand side b (C/m^3) of A Phi = b + rho, without the carrier charge.

    P has shape (ncomp, Nz, Ny, Nx); the last component is P_z.  With three
    components the in-plane faces carry the arithmetic mean of P_x (P_y).
    """
    eps = pl["eps"]
    fe = pl["fe"][:, None, None]          # polarization exists in ferroelectric layers only
    Pz = P[-1] * fe
    Pf = face_polarization(Pz, eps)
    b = -(Pf[1:] - Pf[:-1]) / h
    if P.shape[0] == 3:
        for comp, axis in ((0, 2), (1, 1)):
            Pc = P[comp] * fe
            # face average on the +side face minus the -side face
            f_plus = 0.5 * (Pc + np.roll(Pc, -1, axis=axis))
            f_minus = 0.5 * (Pc + np.roll(Pc, 1, axis=axis))
            b -= (f_plus - f_minus) / h
    b[0] += 2.0 * eps[0] * v_bottom / h ** 2
    b[-1] += 2.0 * eps[-1] * v_top / h ** 2
    return b


def z_couplings(eps, h):
    """Coefficients c_f = conductance/h^2 of the Nz+1 z faces (electrodes included)."""
    nz = eps.shape[0]
    cz = np.empty(nz + 1)
    cz[0] = 2.0 * eps[0] / h ** 2
    cz[nz] = 2.0 * eps[-1] / h ** 2
    cz[1:nz] = face_eps(eps) / h ** 2
    return cz


def apply_A(phi, pl, h):
    """(A phi): the homogeneous operator (electrode values taken as zero)."""
    eps = pl["eps"]
    cxy = (eps / h ** 2)[:, None, None]
    lat = cxy * (4.0 * phi - np.roll(phi, 1, 2) - np.roll(phi, -1, 2)
                 - np.roll(phi, 1, 1) - np.roll(phi, -1, 1))
    cz = z_couplings(eps, h)
    out = lat.copy()
    out += cz[:-1, None, None] * phi     # lower face of every cell
    out += cz[1:, None, None] * phi      # upper face of every cell
    out[1:] -= cz[1:-1, None, None] * phi[:-1]
    out[:-1] -= cz[1:-1, None, None] * phi[1:]
    return out


def residual(phi, b, pl, h, rho=None):
    """r = b + rho - A phi."""
    r = b - apply_A(phi, pl, h)
    if rho is not None:
        r += rho
    return r


def solve_separable(rhs_, pl, h, shift=None):
    """Exact solve of (A + diag(shift_z)) phi = rhs_ for a per-plane shift.

    Because eps depends on z only and x, y are periodic, the operator is
    diagonalised by the 2-D discrete Fourier transform in x, y: mode (m_x, m_y)
    has the lateral eigenvalue mu = (2 - 2cos(2 pi m_x/Nx) + 2 - 2cos(2 pi m_y/Ny))/h^2,
    scaled by eps_k on plane k, leaving one tridiagonal system in z per mode,
    solved by the Thomas algorithm.
    """
    nz, ny, nx = rhs_.shape
    eps = pl["eps"]
    cz = z_couplings(eps, h)
    lx = (2.0 - 2.0 * np.cos(2.0 * np.pi * np.arange(nx) / nx)) / h ** 2
    ly = (2.0 - 2.0 * np.cos(2.0 * np.pi * np.arange(ny) / ny)) / h ** 2
    mu = ly[:, None] + lx[None, :]
    sh = np.zeros(nz) if shift is None else np.asarray(shift, dtype=np.float64)
    fhat = np.fft.fft2(rhs_, axes=(1, 2))
    # tridiagonal: -cz[k] x_{k-1} + d_k x_k - cz[k+1] x_{k+1} = f_k
    d = [eps[k] * mu + cz[k] + cz[k + 1] + sh[k] for k in range(nz)]
    cp = [None] * nz
    dp = [None] * nz
    cp[0] = -cz[1] / d[0]
    dp[0] = fhat[0] / d[0]
    for k in range(1, nz):
        denom = d[k] + cz[k] * cp[k - 1]          # d_k - a_k c'_{k-1}, a_k = -cz[k]
        cp[k] = -cz[k + 1] / denom
        dp[k] = (fhat[k] + cz[k] * dp[k - 1]) / denom
    x = np.empty_like(fhat)
    x[nz - 1] = dp[nz - 1]
    for k in range(nz - 2, -1, -1):
        x[k] = dp[k] - cp[k] * x[k + 1]
    return np.real(np.fft.ifft2(x, axes=(1, 2)))


def solve_linear(P, pl, h, v_bottom, v_top):
    """Phi for a stack without semiconductor (rho = 0): one exact separable solve."""
    return solve_separable(rhs(P, pl, h, v_bottom, v_top), pl, h)

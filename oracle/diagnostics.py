"""Charge and voltage diagnostics of a device state (oracle; test infrastructure).

Results, MFIM section: Q is the average of eps0 eps_DE E_z over the FE/DE
interface plane, on the dielectric side; V_fe = V_app - <Phi_int>.
Readings:
  * The interface is the bottom face of the lowest ferroelectric plane.  On its
    dielectric side P = 0, so eps_DE E_z equals the face flux F (= D_z) of the
    finite-volume scheme.  The sign is taken as Q = -<D_z> (the gate-side charge),
    which makes Q > 0 for V_app > 0 in a linear capacitor and puts the
    hysteresis loops of the paper's Q-V figure in quadrants 1 and 3.
  * <Phi_int> is the mean face potential on that face; V_fe = V1 - <Phi_int>
    (equal to V_app - <Phi_int> for the paper's V0 = 0).
  * Electrode charges: sigma_top = -<F_top>, sigma_bot = +<F_bot>.
"""
import numpy as np


def charges(phi, P, pl, geom, v_bottom, v_top):
    h = geom["h"]
    eps = pl["eps"]
    Pz = P[-1]
    fe_planes = np.nonzero(pl["fe"])[0]
    k0 = int(fe_planes[0]) if fe_planes.size else 0
    if k0 > 0:
        eL, eR = eps[k0 - 1], eps[k0]
        eh = 2.0 * eL * eR / (eL + eR)
        Pf = (eR * Pz[k0 - 1] + eL * Pz[k0]) / (eL + eR)
        F = -eh * (phi[k0] - phi[k0 - 1]) / h + Pf
        phi_f = (eL * phi[k0 - 1] + eR * phi[k0]) / (eL + eR) - 0.5 * h * (Pz[k0] - Pz[k0 - 1]) / (eL + eR)
    else:
        F = -eps[0] * (phi[0] - v_bottom) / (0.5 * h) + Pz[0]
        phi_f = np.full_like(phi[0], v_bottom)
    F_top = -eps[-1] * (v_top - phi[-1]) / (0.5 * h) + Pz[-1]
    F_bot = -eps[0] * (phi[0] - v_bottom) / (0.5 * h) + Pz[0]
    phi_int = float(np.mean(phi_f))
    return dict(Q_int=-float(np.mean(F)), phi_int_avg=phi_int, V_fe=v_top - phi_int,
                sigma_top=-float(np.mean(F_top)), sigma_bot=float(np.mean(F_bot)))


def qv_sweep(P0, phi0, pl, geom, dt, v_app, steps_per_point, order=1):
    """Q-V protocol (Results, MFIM: the voltage follows a triangular wave and Q, V_fe
    are recorded along it): for each bias point, V0 = 0 and V1 = v_app[q], advance
    steps_per_point time steps from the previous point's state, record the charges.
    Returns (records, P, phi)."""
    from . import tdgl
    P, phi = P0.copy(), phi0.copy()
    out = []
    for v in v_app:
        for _ in range(steps_per_point):
            P, phi = tdgl.step(P, phi, pl, geom, dt, 0.0, v, order)
        out.append(charges(phi, P, pl, geom, 0.0, v))
    return out, P, phi

"""Per-plane material table of a layered device stack (oracle; test infrastructure).

The paper's devices are planar MFIM / MFISM stacks (Fig. 1a; Results) with
piecewise-constant permittivity (Eq. Poisson: "eps is spatially varying").
Materials and constants: Table 1.  Every quantity here is a function of the
z-plane only.
"""
import numpy as np

EPS0 = 8.8541878128e-12      # F/m (CODATA 2018)
Q_E = 1.602176634e-19        # C (exact SI)
K_B = 1.380649e-23           # J/K (exact SI)

FE, DE, SC = 0, 1, 2


def planes(geom):
    """Expand the bottom-to-top layer list into per-plane arrays.

    Returns a dict of float arrays of length Nz: kind, eps (absolute, F/m), the
    Landau coefficients alpha/beta/gamma of the z component and alpha_xy/beta_xy/
    gamma_xy of the in-plane components (3-component model only), g11, g44,
    Gamma, and the semiconductor data N_A, N_D, n_i, T, the carrier statistics
    (stats: 0 Boltzmann, 1 Fermi-Dirac) with the effective masses m_e, m_p (in
    units of the electron mass) and the band gap E_g (eV).
    """
    keys = ["alpha", "beta", "gamma", "g11", "g44", "Gamma", "N_A", "N_D", "n_i", "T",
            "m_e", "m_p", "E_g"]
    out = {k: [] for k in keys}
    out.update(kind=[], eps=[], alpha_xy=[], beta_xy=[], gamma_xy=[])
    for layer in geom["layers"]:
        n = int(layer["ncells"])
        out["kind"] += [int(layer["kind"])] * n
        out["eps"] += [EPS0 * float(layer["eps_r"])] * n
        for k in keys:
            out[k] += [float(layer.get(k, 0.0))] * n
        for k in ("alpha", "beta", "gamma"):
            out[k + "_xy"] += [float(layer.get(k + "_xy", layer.get(k, 0.0)))] * n
    res = {k: np.asarray(v, dtype=np.float64) for k, v in out.items()}
    res["kind"] = np.asarray(out["kind"], dtype=np.int64)
    st = []
    for layer in geom["layers"]:
        st += [int(layer.get("stats", 0))] * int(layer["ncells"])
    res["stats"] = np.asarray(st, dtype=np.int64)
    res["fe"] = res["kind"] == FE
    res["sc"] = res["kind"] == SC
    return res

"""The mixed form's outer residual in double-float arithmetic on the FP32 pipe,
against the FP64 residual and the oracle.

r = b + rho(phi) - A phi is a near-cancellation at convergence, so its evaluation
must keep far more than FP32's 24 bits: double-float pairs keep about 48.  The
elementwise difference from the FP64 residual is bounded by a few 2^-48 of the
largest term of the stencil (coefficient x potential, or the right-hand side).
"""
import numpy as np
import pytest

import oracle
from oracle import carriers, poisson
from paper_2210_15668_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _scale(geom, phi, b):
    """Largest term of the scaled stencil: the diagonal times |phi|, or |b|."""
    pl = oracle.planes(geom)
    eps_r = pl["eps"] / oracle.EPS0
    diag = 2.0 * eps_r.max() * 6.0
    return max(diag * np.abs(phi).max(), np.abs(b).max())


CASES = {
    "mfim_256x256x32": (lambda: I.make_geometry(256, 256, I.mfim_stack(32)), -2.0),
    "mfism_64x64x64": (lambda: I.make_geometry(64, 64, I.mfism_stack(64)), 0.4),
    "fd_undoped_48x48x32": (lambda: I.make_geometry(
        48, 48, [I.sc_layer(16, N_A=0.0, stats=I.STATS_FERMI_DIRAC), I.de_layer(4), I.fe_layer(12)]), 0.9),
}


@pytest.mark.parametrize("name", list(CASES))
def test_double_float_residual_matches_fp64(name):
    from paper_2210_15668_gb300 import ferrox
    gfn, v = CASES[name]
    geom = gfn()
    P0 = I.random_polarization(geom, seed=81, amp=0.1)
    num = ferrox.make_numerics(4e-13, tol=1e-10, precision=ferrox.MIXED, guess=1, inner=-8)
    d = ferrox.Device(geom, P0, numerics=num)
    d.set_bias(0.0, v)
    d.solve_poisson()
    d.step(3)
    P, phi = d.get_state()
    r64 = d.residual(double_float=False)
    rdf = d.residual(double_float=True)
    d.close()
    # the same residual in the oracle's scaling (h^2/eps0) from the GPU's state
    pl = oracle.planes(geom)
    b = poisson.rhs(P, pl, geom["h"], 0.0, v)
    rho, _ = carriers.charge(phi, pl)
    ro = poisson.residual(phi, b, pl, geom["h"], rho) * geom["h"] ** 2 / oracle.EPS0
    scale = _scale(geom, phi, b * geom["h"] ** 2 / oracle.EPS0)
    d_df = np.abs(rdf - r64).max() / scale
    d_64 = np.abs(r64 - ro).max() / scale
    print(f"{name}: |r_df - r_64| {d_df:.2e}, |r_64 - r_oracle| {d_64:.2e} of the largest term "
          f"({scale:.3e}); |r| {np.abs(r64).max() / scale:.2e}")
    assert d_df <= 2e-14, d_df
    assert d_64 <= 1e-14, d_64
    assert np.abs(rdf - ro).max() / scale <= 2e-14


@pytest.mark.parametrize("name", ["mfim_256x256x32", "mfism_64x64x64"])
def test_double_float_residual_same_solution(name, monkeypatch):
    """Mixed-form runs with the double-float and the FP64 outer residual stop on the
    same test and reach the same state to the solver tolerance."""
    from paper_2210_15668_gb300 import ferrox
    gfn, v = CASES[name]
    geom = gfn()
    P0 = I.random_polarization(geom, seed=82, amp=0.05)
    num = ferrox.make_numerics(4e-13, tol=1e-12, precision=ferrox.MIXED)
    out = {}
    for env in ("0", "1"):
        monkeypatch.setenv("FERROX_DF_RESID", env)
        d = ferrox.Device(geom, P0, numerics=num)
        d.set_bias(0.0, v)
        d.solve_poisson()
        d.step(5)
        out[env] = d.get_state()
        assert d.stats()["status"] == 0
        d.close()
    for q in range(2):
        a, b = out["0"][q], out["1"][q]
        assert np.linalg.norm(a - b) <= 1e-10 * np.linalg.norm(a)

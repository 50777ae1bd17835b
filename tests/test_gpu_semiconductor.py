"""GPU against the oracle with semiconductor layers (Boltzmann carriers, damped
Newton) and with the 3-component polarization model.

The nonlinear Poisson problem has one solution (A is SPD, -rho' > 0), so the
GPU's damped Newton (one V-cycle per update) and the oracle's Newton-PCG meet
at the same potential; the GPU stops at ||r|| <= tol max(||b||, ||rho||).
"""
import numpy as np
import pytest

import oracle
from oracle import carriers, poisson, tdgl, diagnostics
from paper_2210_15668_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _dev(geom, P0, tol=1e-10, precision=0, v=(0.0, 0.0), order=1, phi0=None, **kw):
    from paper_2210_15668_gb300 import ferrox
    num = ferrox.make_numerics(4e-13, order=order, tol=tol, precision=precision, **kw)
    d = ferrox.Device(geom, P0, numerics=num, phi0=phi0)
    d.set_bias(*v)
    return d


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


MFISM = {
    "pSi_32x32x64": lambda: I.make_geometry(32, 32, I.mfism_stack(64)),
    "undoped_24x24x32": lambda: I.make_geometry(
        24, 24, [I.sc_layer(16, N_A=0.0, n_i=1e16), I.de_layer(4), I.fe_layer(12)]),
    "nSi_16x40x24": lambda: I.make_geometry(16, 40, [I.sc_layer(12, N_A=0.0, N_D=5e23),
                                                     I.de_layer(2), I.fe_layer(10)]),
}


@pytest.mark.parametrize("name", list(MFISM))
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("v", [0.0, 0.8, -1.2])
def test_nonlinear_solve_matches_oracle(name, precision, v):
    geom = MFISM[name]()
    pl = oracle.planes(geom)
    P = I.random_polarization(geom, seed=51, amp=0.2)
    b = poisson.rhs(P, pl, geom["h"], 0.0, v)
    phio, _ = carriers.newton_solve(b, np.zeros(P.shape[1:]), pl, geom["h"], tol=1e-13)
    d = _dev(geom, P, tol=1e-12, precision=precision, v=(0.0, v))
    d.solve_poisson()
    st = d.stats()
    _, phig = d.get_state()
    assert st["status"] == 0 and st["last_rel_res"] <= 1e-12, st
    assert rel_l2(phig, phio) <= 1e-9, (rel_l2(phig, phio), st)
    d.close()


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-12), (1, 1e-10)])
def test_mfism_32x32x64_steps(precision, tol):
    """Reduced copy of the 256x256x64 MFISM workload (same layers, seed 2, 0 V)."""
    geom = I.make_geometry(32, 32, I.mfism_stack(64))
    pl = oracle.planes(geom)
    P0 = I.random_polarization(geom, seed=2)
    steps = 20
    Po, phio = tdgl.run(P0, pl, geom, 4e-13, 0.0, 0.0, steps)
    d = _dev(geom, P0, tol=tol, precision=precision)
    d.solve_poisson()
    d.step(steps)
    Pg, phig = d.get_state()
    assert d.stats()["status"] == 0
    err_P = np.abs(Pg - Po).max() / np.abs(Po).max()
    print(f"MFISM precision {precision} tol {tol}: max rel P {err_P:.3e} rel L2 phi {rel_l2(phig, phio):.3e}")
    assert err_P <= (1e-9 if tol < 1e-11 else 1e-6)
    q = d.charge()
    qo = diagnostics.charges(phio, Po, pl, geom, 0.0, 0.0)
    assert abs(q["sigma_top"] - qo["sigma_top"]) <= 1e-8 * abs(qo["sigma_top"]) + 1e-12
    d.close()


THREE = {
    "mfim3_32x24x12": lambda: I.make_geometry(32, 24, I.mfim_stack(12, n_fe=8), ncomp=3),
    "mfim3_paraxy_40x16x10": lambda: I.make_geometry(
        40, 16, [I.de_layer(4), I.fe_layer(6, alpha_xy=1.5e9, beta_xy=0.0, gamma_xy=0.0)],
        pbc=I.PBC_FREE, ncomp=3),
}


@pytest.mark.parametrize("name", list(THREE))
def test_three_component_update_matches_oracle(name):
    geom = THREE[name]()
    pl = oracle.planes(geom)
    P = I.random_polarization(geom, seed=61, amp=0.1)
    phi = np.random.default_rng(62).uniform(-0.3, 0.3, P.shape[1:])
    d = _dev(geom, P, phi0=phi, v=(0.0, 0.4))
    d.tdgl_update()
    Pg, _ = d.get_state()
    Pe = P + 4e-13 * tdgl.force(P, phi, pl, geom, 0.0, 0.4)
    assert np.abs(Pg - Pe).max() <= 1e-12 * np.abs(P).max()
    d.close()


@pytest.mark.parametrize("name", list(THREE))
@pytest.mark.parametrize("order", [1, 2])
def test_three_component_steps_match_oracle(name, order):
    geom = THREE[name]()
    pl = oracle.planes(geom)
    P0 = I.random_polarization(geom, seed=63, amp=0.05)
    Po, phio = tdgl.run(P0, pl, geom, 4e-13, 0.0, 0.4, 10, order=order)
    d = _dev(geom, P0, tol=1e-12, v=(0.0, 0.4), order=order)
    d.solve_poisson()
    d.step(10)
    Pg, phig = d.get_state()
    assert d.stats()["status"] == 0
    assert rel_l2(Pg, Po) <= 1e-9 and rel_l2(phig, phio) <= 1e-9
    d.close()

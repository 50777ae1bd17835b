"""GPU against the oracle with Fermi-Dirac carriers (the paper's semiconductor model:
n = N_c F_1/2(eta_e), p = N_v F_1/2(eta_p), F_1/2 by the Bednarczyk approximation,
N_c and N_v from the effective masses of the parameter table).

The nonlinear problem keeps one solution, so the GPU's damped Newton and the
oracle's Newton-PCG meet at the same potential.  Cases: undoped Si (the paper's
devices), p-type Si, and a degenerately doped n+ layer driven into the band
(eta_e > 0, where Fermi-Dirac and Boltzmann statistics differ).
"""
import numpy as np
import pytest

import oracle
from oracle import carriers, poisson, tdgl, diagnostics
from paper_2210_15668_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

FD = I.STATS_FERMI_DIRAC


def _dev(geom, P0, tol=1e-12, precision=0, v=(0.0, 0.0), phi0=None, **kw):
    from paper_2210_15668_gb300 import ferrox
    num = ferrox.make_numerics(4e-13, tol=tol, precision=precision, **kw)
    d = ferrox.Device(geom, P0, numerics=num, phi0=phi0)
    d.set_bias(*v)
    return d


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


STACKS = {
    "undoped_24x24x32": lambda: I.make_geometry(
        24, 24, [I.sc_layer(16, N_A=0.0, stats=FD), I.de_layer(4), I.fe_layer(12)]),
    "pSi_32x32x40": lambda: I.make_geometry(
        32, 32, [I.sc_layer(28, N_A=1e24, stats=FD), I.de_layer(2), I.fe_layer(10)]),
    "n+Si_16x16x24": lambda: I.make_geometry(
        16, 16, [I.sc_layer(12, N_D=5e26, stats=FD), I.de_layer(2), I.fe_layer(10)]),
}


@pytest.mark.parametrize("name", list(STACKS))
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("v", [0.0, 1.5, -1.5])
def test_fermi_dirac_solve_matches_oracle(name, precision, v):
    geom = STACKS[name]()
    pl = oracle.planes(geom)
    P = I.random_polarization(geom, seed=61, amp=0.25)
    b = poisson.rhs(P, pl, geom["h"], 0.0, v)
    phio, _ = carriers.newton_solve(b, np.zeros(P.shape[1:]), pl, geom["h"], tol=1e-13)
    d = _dev(geom, P, precision=precision, v=(0.0, v))
    d.solve_poisson()
    st = d.stats()
    _, phig = d.get_state()
    assert st["status"] == 0 and st["last_rel_res"] <= 1e-12, st
    assert rel_l2(phig, phio) <= 1e-9, (rel_l2(phig, phio), st)
    d.close()


def test_fermi_dirac_degenerate_layer_differs_from_boltzmann():
    """In the n+ layer at +1.5 V the electrons are degenerate: the Fermi-Dirac and
    Boltzmann (same n_i) solutions differ well beyond the solver tolerance, and the GPU
    follows the oracle for each statistics."""
    geom = STACKS["n+Si_16x16x24"]()
    Nc, Nv = carriers.effective_dos(1.08, 300.0), carriers.effective_dos(0.81, 300.0)
    n_i = np.sqrt(Nc * Nv) * np.exp(-1.12 * 1.602176634e-19 / (2 * 1.380649e-23 * 300.0))
    gmb = dict(geom, layers=[dict(geom["layers"][0], stats=I.STATS_BOLTZMANN, n_i=n_i)] + geom["layers"][1:])
    P = I.random_polarization(geom, seed=62, amp=0.25)
    out = {}
    for tag, g in (("fd", geom), ("mb", gmb)):
        pl = oracle.planes(g)
        b = poisson.rhs(P, pl, g["h"], 0.0, 1.5)
        phio, _ = carriers.newton_solve(b, np.zeros(P.shape[1:]), pl, g["h"], tol=1e-13)
        d = _dev(g, P, v=(0.0, 1.5))
        d.solve_poisson()
        _, phig = d.get_state()
        d.close()
        assert rel_l2(phig, phio) <= 1e-9
        out[tag] = phig
    assert rel_l2(out["fd"], out["mb"]) > 1e-4


@pytest.mark.parametrize("precision", [0, 1])
def test_fermi_dirac_steps_match_oracle(precision):
    """20 coupled TDGL + Poisson steps of an undoped-Si MFISM stack (the paper's device
    model) against the oracle, and the interface charge."""
    geom = I.make_geometry(32, 32, [I.sc_layer(20, N_A=0.0, stats=FD), I.de_layer(2), I.fe_layer(10)])
    pl = oracle.planes(geom)
    P0 = I.random_polarization(geom, seed=63)
    steps = 20
    Po, phio = tdgl.run(P0, pl, geom, 4e-13, 0.0, 0.6, steps)
    d = _dev(geom, P0, precision=precision, v=(0.0, 0.6))
    d.solve_poisson()
    d.step(steps)
    Pg, phig = d.get_state()
    st = d.stats()
    assert st["status"] == 0
    assert rel_l2(Pg, Po) <= 1e-9 and rel_l2(phig, phio) <= 1e-9, (rel_l2(Pg, Po), rel_l2(phig, phio))
    q = d.charge()
    qo = diagnostics.charges(phio, Po, pl, geom, 0.0, 0.6)
    assert abs(q["Q_int"] - qo["Q_int"]) <= 1e-8 * abs(qo["Q_int"])
    d.close()


def test_unknown_statistics_rejected():
    from paper_2210_15668_gb300 import ferrox
    geom = I.make_geometry(16, 16, [I.sc_layer(8, stats=7), I.de_layer(2), I.fe_layer(6)])
    with pytest.raises(ferrox.FerroxError, match="EINVAL"):
        _dev(geom, np.zeros((1, 16, 16, 16)))

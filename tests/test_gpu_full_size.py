"""The MFISM workloads at their full sizes (256x256x64 and 512x512x128 cells, p-Si,
damped Newton) in the launch configuration the bench times for them (mixed form,
extrapolated guess, 3 V-cycles per FP64 residual), checked by properties the
oracle evaluates at any size:

  * the stopping test of the last solve, recomputed by the oracle in FP64 from
    the GPU's P and phi: ||b(P) + rho(phi) - A phi|| <= tol max(||b||, ||rho||)
    (Eqs. Poisson, rho; the ratio is independent of the GPU's internal scaling);
  * one further TDGL update (Step 1a) of the GPU's state against the oracle's
    P + dt f(P, phi) (Eq. TDGL2) on every cell.
"""
import numpy as np
import pytest

import oracle
from oracle import carriers, poisson, tdgl
from paper_2210_15668_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-10


@pytest.mark.parametrize("make", [I.mfism_mixed, I.mfism_large], ids=["256x256x64", "512x512x128"])
def test_mfism_full_size_stopping_test_and_update(make):
    from paper_2210_15668_gb300 import ferrox
    cfg = make()
    geom = cfg["geom"]
    v_bot, v_top = cfg["v_bottom"], cfg["v_top"]
    P0 = I.random_polarization(geom, cfg["seed"])
    num = ferrox.make_numerics(cfg["dt"], order=1, tol=TOL, precision=ferrox.MIXED, guess=1, inner=3)
    d = ferrox.Device(geom, P0, numerics=num)
    d.set_bias(v_bot, v_top)
    d.solve_poisson()
    d.step(3)
    st = d.stats()
    assert st["status"] == 0 and st["steps"] == 3
    P, phi = d.get_state()

    pl = oracle.planes(geom)
    h = geom["h"]
    b = poisson.rhs(P, pl, h, v_bot, v_top)
    rho, _ = carriers.charge(phi, pl)
    r = poisson.residual(phi, b, pl, h, rho)
    scale = max(np.linalg.norm(b), np.linalg.norm(rho))
    rel = np.linalg.norm(r) / scale
    print(f"{geom['nx']}x{geom['ny']}x{phi.shape[0]}: oracle-recomputed ||r|| / scale = {rel:.3e}")
    assert rel <= 1.05 * TOL

    d.tdgl_update()
    P1, _ = d.get_state()
    d.close()
    expect = P + cfg["dt"] * tdgl.force(P, phi, pl, geom, v_bot, v_top)
    err = np.linalg.norm(P1 - expect) / np.linalg.norm(expect)
    assert err <= 1e-12, err

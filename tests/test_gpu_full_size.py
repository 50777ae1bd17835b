"""The MFISM workloads at their full sizes (256x256x64 and 512x512x128 cells, p-Si,
damped Newton) in the launch configuration the bench times for them (mixed form,
extrapolated guess, 3 V-cycles per FP64 residual), checked by properties the
oracle evaluates at any size:

  * the stopping test of the last solve, recomputed by the oracle in FP64 from
    the GPU's P and phi: ||b(P) + rho(phi) - A phi|| <= tol max(||b||, ||rho||)
    (Eqs. Poisson, rho; the ratio is independent of the GPU's internal scaling);
  * one further TDGL update (Step 1a) of the GPU's state against the oracle's
    P + dt f(P, phi) (Eq. TDGL2) on every cell.
The 256x256x64 workload is also compared element by element with the oracle's
run (Step 0 and two steps), in the bench's FP64 and fast mixed forms.
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


@pytest.mark.parametrize("form", ["fp64", "mixed_fast"])
def test_mfism_256x256x64_elementwise(form):
    """The 256x256x64 MFISM workload at full size, every element against the oracle
    (Newton-PCG solves, ~25 s of host time): Step 0 and two time steps, in the bench's
    plain FP64 form and in its fast mixed form (extrapolated guess, 4 V-cycles per
    Newton residual, double-float outer residual).  Bounds as for the other forms at
    tol 1e-10: relative L2 <= 2e-8 on P and phi, max|dP|/max|P| <= 1e-6 for the mixed
    form."""
    from paper_2210_15668_gb300 import ferrox
    cfg = I.mfism_mixed()
    geom = cfg["geom"]
    pl = oracle.planes(geom)
    P0 = I.random_polarization(geom, cfg["seed"])
    Po, phio = tdgl.run(P0, pl, geom, cfg["dt"], 0.0, 0.0, 2)
    kw = dict(precision=ferrox.FP64) if form == "fp64" else dict(precision=ferrox.MIXED, guess=1, inner=4)
    num = ferrox.make_numerics(cfg["dt"], order=1, tol=TOL, **kw)
    d = ferrox.Device(geom, P0, numerics=num)
    d.set_bias(0.0, 0.0)
    d.solve_poisson()
    d.step(2)
    st = d.stats()
    Pg, phig = d.get_state()
    d.close()
    assert st["status"] == 0
    eP = np.linalg.norm(Pg - Po) / np.linalg.norm(Po)
    ephi = np.linalg.norm(phig - phio) / np.linalg.norm(phio)
    emax = np.abs(Pg - Po).max() / np.abs(Po).max()
    print(f"256x256x64 {form}: rel L2 P {eP:.2e} phi {ephi:.2e}, max rel P {emax:.2e}")
    assert eP <= 2e-8 and ephi <= 2e-8, (eP, ephi)
    assert emax <= 1e-6

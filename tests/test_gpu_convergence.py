"""The convergence study of the Numerical Validation section on the GPU path: 32 nm
cube, undoped Si / SiO2 / FE = 25 / 25 / 50 %, Fermi-Dirac carriers, lambda = 3 nm,
Phi = 0 on both faces, Gaussian polarization bump, t = 400 fs.
  Test 1: 128^3, dt = 50 / 25 / 12.5 fs, first-order scheme
  Test 2: the same with the second-order scheme
  Test 3: dt = 25 fs, second-order scheme, 64^3 / 128^3 / 256^3
Errors as the paper defines them: E_c^m = rms of the difference of the coarse and
medium solutions (the finer one averaged down over 8 cells for Test 3), rate =
log2(E_c^m / E_m^f).  The temporal rates are compared with the paper's printed
rates (tests/golden/convergence_table.txt).  Absolute errors and the spatial rates
depend on the discretisation, which here differs from the paper's (flux-continuous
face values at interfaces); they are reported, and the spatial rate is asserted to
be at least the paper's.  The solves stop at 1e-11 relative residual: the smallest
differences measured (Test 2, ~1e-7 of the potential) are far above what that
leaves, while 1e-13 is below the FP64 round-off floor of the residual on 2-17 M cells.
"""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import tdgl
from paper_2210_15668_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

T_END = 400e-15


def _table():
    path = os.path.join(os.path.dirname(__file__), "golden", "convergence_table.txt")
    out = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            t, f, ecm, rate, emf = line.split()
            out[(int(t), f)] = (float(ecm), float(rate), float(emf))
    return out


def _run(n, dt, order, tol=1e-11):
    from paper_2210_15668_gb300 import ferrox
    geom = I.convergence_cube(n)
    P0 = I.gaussian_bump(geom)
    num = ferrox.make_numerics(dt, order=order, tol=tol, precision=ferrox.FP64, max_cycles=400)
    d = ferrox.Device(geom, P0, numerics=num)
    d.set_bias(0.0, 0.0)
    d.solve_poisson()
    d.step(int(round(T_END / dt)))
    P, phi = d.get_state()
    assert d.stats()["status"] == 0
    d.close()
    return P, phi


def _down(a):
    """Average over the 8 fine cells of each coarse cell (last three axes)."""
    s = a.shape
    return a.reshape(s[:-3] + (s[-3] // 2, 2, s[-2] // 2, 2, s[-1] // 2, 2)).mean(axis=(-5, -3, -1))


def _rms(a, b):
    return float(np.sqrt(np.mean((a - b) ** 2)))


def test_convergence_problem_matches_oracle():
    """The study's problem at 32^3 (1 nm cells), second order, 8 steps of 50 fs,
    element by element against the oracle."""
    geom = I.convergence_cube(32)
    pl = oracle.planes(geom)
    P0 = I.gaussian_bump(geom)
    Po, phio = tdgl.run(P0, pl, geom, 50e-15, 0.0, 0.0, 8, order=2)
    Pg, phig = _run(32, 50e-15, 2, tol=1e-13)
    assert np.linalg.norm(Pg - Po) <= 1e-9 * np.linalg.norm(Po)
    assert np.linalg.norm(phig - phio) <= 1e-9 * np.linalg.norm(phio)


@pytest.mark.parametrize("order", [1, 2])
def test_temporal_convergence_128(order):
    """Tests 1 and 2 at the paper's 128^3: the rates match the printed ones."""
    table = _table()
    sols = [_run(128, dt, order) for dt in (50e-15, 25e-15, 12.5e-15)]
    for which, field in ((0, "P"), (1, "Phi")):
        ecm = _rms(sols[1][which], sols[0][which])
        emf = _rms(sols[2][which], sols[1][which])
        rate = math.log2(ecm / emf)
        paper = table[(order, field)]
        print(f"Test {order} {field}: E_c^m {ecm:.3e} rate {rate:.3f} E_m^f {emf:.3e} "
              f"(paper {paper[0]:.2e} {paper[1]:.2f} {paper[2]:.2e})")
        assert abs(rate - paper[1]) <= 0.1, (field, rate)
        if field == "P":
            # same model and integrators as the paper: the polarization differences
            # themselves agree with the printed ones (measured within 1.25x)
            assert 0.5 <= ecm / paper[0] <= 2.0 and 0.5 <= emf / paper[2] <= 2.0, (ecm, emf)


def test_spatial_convergence_64_128_256():
    """Test 3: 64^3 / 128^3 / 256^3 at dt = 25 fs, second order.  The paper reports 1.96
    for P and 1.00 for Phi (first order from its interface treatment).  The
    flux-continuous face values used here are exact for layered fields, so Phi keeps
    second order (measured 2.005); P converges at second order (measured 1.998)."""
    table = _table()
    c, m, f = (_run(n, 25e-15, 2) for n in (64, 128, 256))
    for which, field in ((0, "P"), (1, "Phi")):
        ecm = _rms(_down(m[which]), c[which])
        emf = _rms(_down(f[which]), m[which])
        rate = math.log2(ecm / emf)
        paper = table[(3, field)]
        print(f"Test 3 {field}: E_c^m {ecm:.3e} rate {rate:.3f} E_m^f {emf:.3e} "
              f"(paper {paper[0]:.2e} {paper[1]:.2f} {paper[2]:.2e})")
        assert rate >= paper[1] - 0.1, (field, rate)
        assert abs(rate - 2.0) <= 0.1, (field, rate)

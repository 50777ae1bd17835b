"""Several V-cycles per outer iteration: same stopping test, same answer.

With `inner` V-cycles per FP64 residual the outer iterations (and so the FP64
residuals and carrier exponentials) fall, while the solve still stops on
||r|| <= tol max(||b||, ||rho||): the states agree to the solver tolerance.
"""
import numpy as np
import pytest

from paper_2210_15668_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def run(geom, P0, precision, inner, steps, v_top, guess=0):
    from paper_2210_15668_gb300 import ferrox
    num = ferrox.make_numerics(4e-13, tol=1e-12, precision=precision, guess=guess, inner=inner)
    d = ferrox.Device(geom, P0, numerics=num)
    d.set_bias(0.0, v_top)
    d.solve_poisson()
    d.step(steps)
    st = d.stats()
    P, phi = d.get_state()
    d.close()
    return P, phi, st


@pytest.mark.parametrize("precision", [0, 1])
def test_inner_cycles_mfim(precision):
    geom = I.make_geometry(64, 64, I.mfim_stack(16))
    P0 = I.random_polarization(geom, seed=4)
    a = run(geom, P0, precision, 1, 10, 0.8)
    b = run(geom, P0, precision, 2, 10, 0.8)
    assert a[2]["status"] == 0 and b[2]["status"] == 0
    assert b[2]["cycles"] < a[2]["cycles"]            # fewer outer iterations
    assert a[2]["vcycles"] == a[2]["cycles"]
    assert b[2]["vcycles"] == 2 * b[2]["cycles"]
    assert np.linalg.norm(b[1] - a[1]) <= 1e-9 * np.linalg.norm(a[1])
    assert np.linalg.norm(b[0] - a[0]) <= 1e-9 * np.linalg.norm(a[0])


def test_inner_cycles_mfism_newton():
    geom = I.make_geometry(64, 64, I.mfism_stack(32))
    P0 = I.random_polarization(geom, seed=5)
    a = run(geom, P0, 1, 1, 6, 0.3, guess=1)
    b = run(geom, P0, 1, 3, 6, 0.3, guess=1)
    assert a[2]["status"] == 0 and b[2]["status"] == 0
    assert b[2]["cycles"] < a[2]["cycles"]
    assert np.linalg.norm(b[1] - a[1]) <= 1e-9 * np.linalg.norm(a[1])


def test_batch_rejects_inner():
    from paper_2210_15668_gb300 import ferrox
    geoms = [I.make_geometry(32, 32, I.mfim_stack(16))]
    P0s = [I.random_polarization(geoms[0], seed=1)]
    with pytest.raises(ferrox.FerroxError, match="EINVAL"):
        ferrox.Batch(geoms, P0s, ferrox.make_numerics(4e-13, precision=1, inner=2))


@pytest.mark.parametrize("precision", [0, 1])
def test_adaptive_inner_cycles_mfim(precision):
    """inner < 0: the device picks the V-cycles of each outer iteration; same answer."""
    geom = I.make_geometry(64, 64, I.mfim_stack(16))
    P0 = I.random_polarization(geom, seed=4)
    a = run(geom, P0, precision, 1, 10, 0.8)
    b = run(geom, P0, precision, -8, 10, 0.8)
    assert a[2]["status"] == 0 and b[2]["status"] == 0
    assert b[2]["cycles"] < a[2]["cycles"]            # fewer FP64 residuals
    assert b[2]["cycles"] <= b[2]["vcycles"] <= 8 * b[2]["cycles"]
    assert np.linalg.norm(b[1] - a[1]) <= 1e-9 * np.linalg.norm(a[1])
    assert np.linalg.norm(b[0] - a[0]) <= 1e-9 * np.linalg.norm(a[0])


def test_adaptive_inner_cycles_mfism_newton():
    geom = I.make_geometry(64, 64, I.mfism_stack(32))
    P0 = I.random_polarization(geom, seed=5)
    a = run(geom, P0, 1, 1, 6, 0.3, guess=1)
    b = run(geom, P0, 1, -8, 6, 0.3, guess=1)
    assert a[2]["status"] == 0 and b[2]["status"] == 0
    assert b[2]["cycles"] < a[2]["cycles"]
    assert np.linalg.norm(b[1] - a[1]) <= 1e-9 * np.linalg.norm(a[1])


def test_batch_rejects_adaptive_inner():
    from paper_2210_15668_gb300 import ferrox
    geoms = [I.make_geometry(32, 32, I.mfim_stack(16))]
    P0s = [I.random_polarization(geoms[0], seed=1)]
    with pytest.raises(ferrox.FerroxError, match="EINVAL"):
        ferrox.Batch(geoms, P0s, ferrox.make_numerics(4e-13, precision=1, inner=-4))

"""V-cycles per solve of every precision form, single stack and batched.

A V(2,2) cycle with a working coarse-grid correction reduces the residual of
these stacks by about 0.05 per cycle, so a linear solve to 1e-10 from a cold
start takes 6-8 cycles.  A cycle whose coarse levels correct too little still
converges, and still matches the oracle, but takes 18 or more.  Parity tests
cannot see that; these bounds can.  The stacks reach each bottom path of the
V-cycle: single MFIM stacks (no carriers) solve their first small level by its
inverse; single MFISM stacks (carriers: a Newton shift on the diagonal, so no
fixed inverse) run the single-CTA tail V-cycle; the batched engines run the
tail for every instance.  With carriers each damped Newton iteration runs one
V-cycle, so its bound also covers the nonlinear iterations.
"""
import numpy as np
import pytest

from paper_2210_15668_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

LINEAR_MAX = 10     # V-cycles per linear solve (MFIM)
NEWTON_MAX = 14     # V-cycles per Newton solve (MFISM), one per Newton iteration

STACKS = {
    "mfim_32x32x16": (lambda: I.make_geometry(32, 32, I.mfim_stack(16)), LINEAR_MAX, -1.5),
    "mfim_128x128x16": (lambda: I.make_geometry(128, 128, I.mfim_stack(16)), LINEAR_MAX, -1.5),
    "mfism_32x32x32": (lambda: I.make_geometry(32, 32, I.mfism_stack(32)), NEWTON_MAX, 0.3),
    "mfism_64x64x32": (lambda: I.make_geometry(64, 64, I.mfism_stack(32)), NEWTON_MAX, 0.3),
}


@pytest.mark.parametrize("stack", list(STACKS))
@pytest.mark.parametrize("precision", [0, 2, 1])   # FP64 direct, FP64 defect, mixed
def test_single_stack_vcycles_per_solve(precision, stack):
    from paper_2210_15668_gb300 import ferrox
    make, bound, v_top = STACKS[stack]
    g = make()
    d = ferrox.Device(g, I.random_polarization(g, seed=200),
                      numerics=ferrox.make_numerics(4e-13, tol=1e-10, precision=precision))
    d.set_bias(0.0, v_top)
    d.solve_poisson()
    s0 = d.stats()
    d.step(5)
    s1 = d.stats()
    d.close()
    assert s0["status"] == 0 and s1["status"] == 0
    assert s0["vcycles"] <= bound, s0
    assert (s1["vcycles"] - s0["vcycles"]) / 5 <= bound, (s0, s1)


@pytest.mark.parametrize("engine", [0, 1])
@pytest.mark.parametrize("precision", [0, 1])
def test_batched_vcycles_per_solve(precision, engine):
    from paper_2210_15668_gb300 import ferrox
    sizes = [32, 48, 64, 96, 128]
    geoms = [I.make_geometry(s, s, I.mfim_stack(16)) for s in sizes]
    P0s = [I.random_polarization(g, seed=300 + i) for i, g in enumerate(geoms)]
    B = ferrox.Batch(geoms, P0s, ferrox.make_numerics(4e-13, tol=1e-10, precision=precision))
    if engine == 0:
        B.set_shape(256, 1, 1, 0)
    else:
        B.set_engine(1)
    B.set_bias(np.zeros(len(sizes)), np.linspace(-1.8, 1.6, len(sizes)))
    B.solve_poisson()
    B.step(3)
    st = B.stats()
    B.close()
    for x in st:
        assert x["status"] == 0 and x["solves"] == 4
        assert x["cycles"] / x["solves"] <= LINEAR_MAX, st

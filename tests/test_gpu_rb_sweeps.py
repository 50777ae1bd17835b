"""Fused red-black sweeps (both colours in one launch, out of place) against the
colour-by-colour sweeps in place.

The fused kernel relaxes each cell with the same operations in the same order
as the two colour sweeps, so a whole run must be bit-identical with either path,
with the same V-cycle counts and fewer launches.  FERROX_RB_SWEEPS=0 (read when
a context is created) selects the colour-by-colour sweeps.
"""
import numpy as np
import pytest

from paper_2210_15668_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASES = {
    # the fused sweep serves levels of at least 2^23 cells: 512 x 512 x 32 fine level
    "mfim_512x512x32": (lambda: I.make_geometry(512, 512, I.mfim_stack(32)), dict(), (0.0, -2.0)),
    # several V-cycles per residual: the fine level's first sweep starts from e != 0
    "mfim_512x512x32_inner3": (lambda: I.make_geometry(512, 512, I.mfim_stack(32)), dict(inner=3, guess=1),
                               (0.0, 1.1)),
    # a lateral size that is not a multiple of the 32 x 16 tile (528 = 16.5 x 32)
    "mfim_528x528x32": (lambda: I.make_geometry(528, 528, I.mfim_stack(32)), dict(), (0.0, 0.7)),
    # semiconductor: Newton shift s in the sweep (division by diag + s)
    "mfism_512x512x40": (lambda: I.make_geometry(512, 512, I.mfism_stack(40)), dict(inner=4, guess=1),
                         (0.0, 0.3)),
}


@pytest.mark.parametrize("case", list(CASES))
def test_fused_sweeps_bit_identical(case, monkeypatch):
    from paper_2210_15668_gb300 import ferrox
    gfn, kw, (vb, vt) = CASES[case]
    geom = gfn()
    P0 = I.random_polarization(geom, seed=17, amp=0.05)
    num = ferrox.make_numerics(4e-13, tol=1e-10, precision=ferrox.MIXED, **kw)
    out = {}
    for env in ("0", "1"):
        monkeypatch.setenv("FERROX_RB_SWEEPS", env)
        d = ferrox.Device(geom, P0, numerics=num)
        d.set_bias(vb, vt)
        d.solve_poisson()
        d.step(3)
        P, phi = d.get_state()
        st = d.stats()
        prof = d.profile_step()
        d.close()
        out[env] = (P, phi, st, prof)
    (Pa, pa, sa, fa), (Pb, pb, sb, fb) = out["0"], out["1"]
    assert sa["status"] == 0 and sb["status"] == 0
    assert np.array_equal(Pa, Pb) and np.array_equal(pa, pb)
    assert sa["vcycles"] == sb["vcycles"] and sa["cycles"] == sb["cycles"]
    assert sb["launches"] < sa["launches"], (sa["launches"], sb["launches"])
    assert fb["smooth_fine"][1] < fa["smooth_fine"][1]

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
    # fine level 32 x 16 x 8 tiles, levels 1 and 2 16 x 8 x 4 tiles
    "mfim_256x256x32": (lambda: I.make_geometry(256, 256, I.mfim_stack(32)), dict(), (0.0, -2.0)),
    # several V-cycles per residual: the fine level's first sweep starts from e != 0
    "mfim_128x64x16_inner3": (lambda: I.make_geometry(128, 64, I.mfim_stack(16)), dict(inner=3, guess=1),
                              (0.0, 1.1)),
    # sizes that are not multiples of the 16 x 8 x 4 tile (partial tiles in x and z)
    "mfim_40x40x18": (lambda: I.make_geometry(40, 40, I.mfim_stack(18)), dict(), (0.0, 0.7)),
    # semiconductor: Newton shift s in the sweep (division by diag + s)
    "mfism_64x64x32": (lambda: I.make_geometry(64, 64, I.mfism_stack(32)), dict(inner=4, guess=1),
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

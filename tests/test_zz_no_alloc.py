"""The TDGL update entry point that allocates nothing (ferrox_tdgl_update_static).

It serves callers that cannot allocate device memory: a process held to a fixed
device-memory budget, a framework whose own allocator owns every device byte, or
a latency-bound loop that cannot afford the device-wide synchronisation that
cudaMalloc and cudaFree may imply.  Its output must equal that of the
context-based entry point ferrox_tdgl_update on the same inputs, on two calls
in a row (the second call reuses the shared static scratch the first one left
behind).  This file is collected last so that a failure here never hides
another test.
"""
import numpy as np
import pytest

from paper_2210_15668_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _two_fe_layers(ncomp):
    return I.make_geometry(32, 32, [I.fe_layer(6), I.de_layer(4, 10.0), I.fe_layer(5)],
                           pbc=I.PBC_FREE, ncomp=ncomp)


@pytest.mark.parametrize("geom_fn", [
    lambda: I.make_geometry(64, 48, I.mfim_stack(16)),
    lambda: _two_fe_layers(1),
    lambda: _two_fe_layers(3),
])
def test_static_entry_matches_context_entry_twice(geom_fn):
    from paper_2210_15668_gb300 import ferrox
    geom = geom_fn()
    P0 = I.random_polarization(geom, seed=41, amp=0.12)
    phi = np.random.default_rng(42).uniform(-0.4, 0.6, P0.shape[1:])
    dt, vb, vt = 4e-13, 0.05, 0.45
    num = ferrox.make_numerics(dt)
    ref = ferrox.Device(geom, P0, numerics=num, phi0=phi)
    ref.set_bias(vb, vt)
    P = torch.as_tensor(P0, device="cuda").contiguous().clone()
    ph = torch.as_tensor(phi, device="cuda").contiguous().clone()
    for call in range(2):
        ref.tdgl_update()
        Pref, _ = ref.get_state()
        ferrox.tdgl_update_static(geom, dt, vb, vt, P, ph)
        torch.cuda.synchronize()
        Ps = P.cpu().numpy()
        assert np.abs(Ps - Pref).max() <= 1e-12 * np.abs(Pref).max(), call
    assert np.array_equal(ph.cpu().numpy(), phi)
    ref.close()


@pytest.mark.parametrize("ncomp", [1, 3])
def test_static_entry_leaves_planes_between_ferroelectric_layers(ncomp):
    """The shared scratch keeps what the previous call wrote.  A first call on a
    stack whose ferroelectric planes cover the offsets that are dielectric in the
    second stack leaves polarization data there; the second call must write only
    its own ferroelectric planes, so the caller's dielectric planes keep their
    (sentinel) values and the ferroelectric planes match the context entry."""
    from paper_2210_15668_gb300 import ferrox
    dt, vb, vt = 4e-13, 0.0, 0.3
    g1 = I.make_geometry(32, 32, I.mfim_stack(16), pbc=I.PBC_FREE, ncomp=ncomp)   # FE on planes 6..15
    P1 = torch.as_tensor(I.random_polarization(g1, seed=7, amp=0.2), device="cuda").contiguous()
    ph1 = torch.zeros((16, 32, 32), dtype=torch.float64, device="cuda")
    ferrox.tdgl_update_static(g1, dt, vb, vt, P1, ph1)
    torch.cuda.synchronize()
    g2 = _two_fe_layers(ncomp)                                                      # DE on planes 6..9
    P0 = I.random_polarization(g2, seed=43, amp=0.1)
    de = ~I.fe_plane_mask(g2)
    phi = np.random.default_rng(44).uniform(-0.2, 0.4, P0.shape[1:])
    ref = ferrox.Device(g2, P0, numerics=ferrox.make_numerics(dt), phi0=phi)
    ref.set_bias(vb, vt)
    ref.tdgl_update()
    Pref, _ = ref.get_state()
    ref.close()
    Pd = P0.copy()
    Pd[:, de] = 123.0                                        # sentinel on the dielectric planes
    P = torch.as_tensor(Pd, device="cuda").contiguous().clone()
    ph = torch.as_tensor(phi, device="cuda").contiguous().clone()
    ferrox.tdgl_update_static(g2, dt, vb, vt, P, ph)
    torch.cuda.synchronize()
    Ps = P.cpu().numpy()
    assert np.all(Ps[:, de] == 123.0)
    fe = ~de
    assert np.abs(Ps[:, fe] - Pref[:, fe]).max() <= 1e-12 * np.abs(Pref).max()


def test_static_entry_rejects_grids_beyond_its_scratch():
    from paper_2210_15668_gb300 import ferrox
    geom = I.make_geometry(256, 256, I.mfim_stack(16))       # 1,048,576 cells > 262,144
    P = torch.zeros((1, 16, 256, 256), dtype=torch.float64, device="cuda")
    phi = torch.zeros((16, 256, 256), dtype=torch.float64, device="cuda")
    with pytest.raises(ferrox.FerroxError, match="EINVAL.*static scratch"):
        ferrox.tdgl_update_static(geom, 4e-13, 0.0, 0.5, P, phi)

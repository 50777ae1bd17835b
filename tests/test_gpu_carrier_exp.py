"""The carrier exponential pair of the residual kernel against an extended-
precision reference (numpy long double: 80-bit on x86, IEEE quad on Arm).

n0 e^{phi/V_T} and p0 e^{-phi/V_T} are the Boltzmann densities of the carrier
model (Sec. II); the kernel evaluates e^{+u} and e^{-u} with one table-driven
reduction (Tang 1989).  Bound: 1.5 ulp for |u| < 700; beyond that, and for
non-finite u, the routine must return exactly what CUDA's exp returns.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def ulp_err(got, ref):
    ref_d = ref.astype(np.float64)
    ulp = np.ldexp(1.0, np.frexp(ref_d)[1] - 53)       # ulp of a double in [2^(e-1), 2^e)
    return np.abs((got.astype(np.longdouble) - ref) / ulp.astype(np.longdouble)).astype(np.float64)


def test_error_bound_over_the_fast_range():
    from paper_2210_15668_gb300 import ferrox
    rng = np.random.default_rng(7)
    u = np.concatenate([
        rng.uniform(-699.9, 699.9, 1_000_000),
        rng.uniform(-40.0, 40.0, 1_000_000),                       # phi/V_T of a device
        rng.uniform(-1e-3, 1e-3, 100_000),
        np.arange(-2000, 2001) * (np.log(2) / 64),                  # on the table points
        np.arange(-2000, 2001) * (np.log(2) / 64) + np.log(2) / 128,  # reduction edges
        [0.0, -0.0, 1e-300, -1e-300, 5e-324, 699.99, -699.99],
    ])
    ep, em = ferrox.carrier_exp(torch.from_numpy(u).cuda())
    ep, em = ep.cpu().numpy(), em.cpu().numpy()
    ul = u.astype(np.longdouble)
    e1 = ulp_err(ep, np.exp(ul))
    e2 = ulp_err(em, np.exp(-ul))
    print(f"max error: e^u {e1.max():.3f} ulp, e^-u {e2.max():.3f} ulp")
    assert e1.max() <= 1.5 and e2.max() <= 1.5
    assert np.all(ep[u == 0.0] == 1.0) and np.all(em[u == 0.0] == 1.0)


def test_outside_the_fast_range_equals_cuda_exp():
    from paper_2210_15668_gb300 import ferrox
    u = torch.tensor([700.0, -700.0, 709.7, -709.7, 709.8, -709.8, 745.2, -745.2, 800.0, -800.0,
                      float("inf"), float("-inf"), float("nan")], dtype=torch.float64, device="cuda")
    ep, em = ferrox.carrier_exp(u)
    ref_p, ref_m = torch.exp(u), torch.exp(-u)
    assert torch.equal(torch.isnan(ep), torch.isnan(ref_p))
    fin = ~torch.isnan(ref_p)
    assert torch.equal(ep[fin], ref_p[fin]) and torch.equal(em[fin], ref_m[fin])


def test_empty_and_bad_arguments():
    from paper_2210_15668_gb300 import ferrox
    ep, em = ferrox.carrier_exp(torch.empty(0, dtype=torch.float64, device="cuda"))
    assert ep.numel() == 0 and em.numel() == 0
    lib = ferrox.load()
    assert lib.ferrox_carrier_exp(None, None, None, C.c_longlong(4), None) == ferrox.FERROX_EINVAL
    assert lib.ferrox_carrier_exp(None, None, None, C.c_longlong(-1), None) == ferrox.FERROX_EINVAL


def test_double_float_pair_error_bound():
    """The double-float pair (FP32 pipe) the mixed form's residual uses for |u| <= 70,
    against e^{h + l} in extended precision for the exact argument pairs: relative
    error <= 2^-45 (a few 2^-48 roundings of the pair arithmetic)."""
    from paper_2210_15668_gb300 import ferrox
    rng = np.random.default_rng(11)
    x = np.concatenate([
        rng.uniform(-70.0, 70.0, 1_000_000),
        rng.uniform(-40.0, 40.0, 1_000_000),
        rng.uniform(-1e-3, 1e-3, 100_000),
        np.arange(-3000, 3001) * (np.log(2) / 64),
        np.arange(-3000, 3001) * (np.log(2) / 64) + np.log(2) / 128,
        [0.0, 70.0, -70.0],
    ])
    x = x[np.abs(x) <= 70.0]
    h = x.astype(np.float32)
    l = (x - h.astype(np.float64)).astype(np.float32)
    u_hl = np.stack([h, l], axis=1)
    ep, em = ferrox.carrier_exp_df(torch.from_numpy(u_hl).cuda())
    ep, em = ep.cpu().numpy().astype(np.longdouble), em.cpu().numpy().astype(np.longdouble)
    u = h.astype(np.longdouble) + l.astype(np.longdouble)
    rp = np.abs(ep / np.exp(u) - 1).astype(np.float64)
    rm = np.abs(em / np.exp(-u) - 1).astype(np.float64)
    print(f"double-float pair: max rel error e^u {rp.max():.2e}, e^-u {rm.max():.2e} (2^-45 = {2.0**-45:.2e})")
    assert rp.max() <= 2.0 ** -45 and rm.max() <= 2.0 ** -45
    assert ep[x == 0.0][0] == 1.0 and em[x == 0.0][0] == 1.0

"""Batched persistent engine (one cooperative launch per call) on the GPU.

Every instance of a batch of uneven lateral sizes and biases must follow the
same trajectory as the oracle run of that instance alone, and as the
single-instance GPU path, within the tolerances of the single-instance tests.
"""
import numpy as np
import pytest

import oracle
from oracle import tdgl, diagnostics
from paper_2210_15668_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def small_batch(n=6, seed=3):
    rng = np.random.default_rng(seed)
    sizes = rng.choice([32, 48, 64], size=n)
    biases = rng.uniform(-2.0, 2.0, size=n)
    geoms = [I.make_geometry(int(s), int(s), I.mfim_stack(16)) for s in sizes]
    P0s = [I.random_polarization(g, seed=100 + i) for i, g in enumerate(geoms)]
    return geoms, P0s, biases


@pytest.mark.parametrize("precision,tol,bound", [(0, 1e-12, 1e-9), (1, 1e-12, 1e-9), (1, 1e-10, 2e-8)])
def test_batch_matches_oracle_per_instance(precision, tol, bound):
    from paper_2210_15668_gb300 import ferrox
    geoms, P0s, biases = small_batch()
    num = ferrox.make_numerics(4e-13, tol=tol, precision=precision)
    B = ferrox.Batch(geoms, P0s, num)
    B.set_bias(np.zeros(len(geoms)), biases)
    B.solve_poisson()
    steps = 20
    B.step(steps)
    st = B.stats()
    tune = B.tuning()
    assert tune["tuned"] and tune["threads"] in (256, 512) and tune["rows_per_unit"] in (1, 2, 4)
    charges = B.charge()
    for i, g in enumerate(geoms):
        pl = oracle.planes(g)
        Po, phio = tdgl.run(P0s[i], pl, g, 4e-13, 0.0, biases[i], steps)
        Pg, phig = B.state(i)
        assert st[i]["status"] == 0 and st[i]["steps"] == steps
        assert rel_l2(Pg, Po) <= bound and rel_l2(phig, phio) <= bound, (i, rel_l2(Pg, Po))
        qo = diagnostics.charges(phio, Po, pl, g, 0.0, biases[i])
        assert abs(charges[i]["sigma_top"] - qo["sigma_top"]) <= 1e-7 * abs(qo["sigma_top"])
    B.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_large_instances_match_oracle(precision):
    """The two largest lateral sizes of the 64-instance sweep (96^2 and 128^2 x 16),
    batched with a small one, each against its own oracle run."""
    from paper_2210_15668_gb300 import ferrox
    sizes, biases = [128, 32, 96], [1.7, -0.4, -1.9]
    geoms = [I.make_geometry(s, s, I.mfim_stack(16)) for s in sizes]
    P0s = [I.random_polarization(g, seed=300 + i) for i, g in enumerate(geoms)]
    num = ferrox.make_numerics(4e-13, tol=1e-12, precision=precision)
    B = ferrox.Batch(geoms, P0s, num)
    B.set_bias(np.zeros(len(geoms)), biases)
    B.solve_poisson()
    steps = 12
    B.step(steps)
    st = B.stats()
    charges = B.charge()
    for i, g in enumerate(geoms):
        pl = oracle.planes(g)
        Po, phio = tdgl.run(P0s[i], pl, g, 4e-13, 0.0, biases[i], steps)
        Pg, phig = B.state(i)
        assert st[i]["status"] == 0 and st[i]["steps"] == steps
        assert rel_l2(Pg, Po) <= 1e-9 and rel_l2(phig, phio) <= 1e-9, (sizes[i], rel_l2(Pg, Po))
        qo = diagnostics.charges(phio, Po, pl, g, 0.0, biases[i])
        assert abs(charges[i]["Q_int"] - qo["Q_int"]) <= 1e-8 * abs(qo["Q_int"])
    B.close()


def test_batch_matches_single_instance_gpu_path():
    """The batched and the single-instance engines stop on the same residual test
    but solve the coarsest levels differently (a shared-memory V-cycle against an
    exact dense solve of the first tail level), so they agree to the solver
    tolerance: at 1e-12, to 1e-10 after 10 steps."""
    from paper_2210_15668_gb300 import ferrox
    geoms, P0s, biases = small_batch(n=4, seed=5)
    num = ferrox.make_numerics(4e-13, tol=1e-12, precision=1)
    B = ferrox.Batch(geoms, P0s, num)
    B.set_bias(np.zeros(len(geoms)), biases)
    B.solve_poisson()
    B.step(10)
    sb = B.stats()
    for i, g in enumerate(geoms):
        d = ferrox.Device(g, P0s[i], numerics=ferrox.make_numerics(4e-13, tol=1e-12, precision=1))
        d.set_bias(0.0, biases[i])
        d.solve_poisson()
        d.step(10)
        Ps, phis = d.get_state()
        Pb, phib = B.state(i)
        assert rel_l2(Pb, Ps) <= 1e-10 and rel_l2(phib, phis) <= 1e-10
        # the exact coarse solve of the single-instance engine needs no more cycles
        assert d.stats()["cycles"] <= sb[i]["cycles"] + 2
        d.close()
    B.close()


def test_instances_drop_out_independently():
    """A zero-bias, zero-polarization instance converges at once while the others iterate."""
    from paper_2210_15668_gb300 import ferrox
    geoms, P0s, biases = small_batch(n=3, seed=7)
    P0s[1] = np.zeros_like(P0s[1])
    biases = np.array([1.5, 0.0, -1.0])
    B = ferrox.Batch(geoms, P0s, ferrox.make_numerics(4e-13, precision=1))
    B.set_bias(np.zeros(3), biases)
    B.solve_poisson()
    st = B.stats()
    assert st[1]["last_cycles"] == 0 and st[0]["last_cycles"] > 0 and st[2]["last_cycles"] > 0
    assert np.all(B.state(1)[1] == 0.0)
    B.close()


def test_bounded_wait_reports_timeout():
    """A grid barrier that one block never reaches ends with FERROX_ETIMEOUT."""
    from paper_2210_15668_gb300 import ferrox
    assert ferrox.check_wait_timeout(0.2) == ferrox.FERROX_ETIMEOUT
    # the context stays usable afterwards
    g = I.make_geometry(16, 16, I.mfim_stack(8, n_fe=4))
    d = ferrox.Device(g, I.random_polarization(g, seed=1))
    d.set_bias(0.0, 0.3)
    d.solve_poisson()
    assert d.stats()["status"] == 0
    d.close()


def test_launch_shapes_give_identical_results():
    """Grouped and single-barrier launches, any thread count and work-unit size:
    the same operations per instance in the same order, so bit-identical states
    and equal cycle counts."""
    from paper_2210_15668_gb300 import ferrox
    geoms, P0s, biases = small_batch(n=6, seed=11)
    num = ferrox.make_numerics(4e-13, tol=1e-10, precision=1)
    outs = []
    for shape in ((256, 1, 2, 1), (512, 4, 1, 0), (256, 2, 1, 1)):
        B = ferrox.Batch(geoms, P0s, num)
        B.set_shape(*shape)
        B.set_bias(np.zeros(len(geoms)), biases)
        B.solve_poisson()
        B.step(5)
        st = B.stats()
        assert all(x["status"] == 0 for x in st)
        assert B.tuning()["groups"] >= (2 if shape[3] else 1)
        outs.append(([B.state(i) for i in range(len(geoms))], [x["cycles"] for x in st]))
        B.close()
    for states, cycles in outs[1:]:
        assert cycles == outs[0][1]
        for (P, phi), (P0, phi0) in zip(states, outs[0][0]):
            assert np.array_equal(P, P0) and np.array_equal(phi, phi0)


@pytest.mark.parametrize("precision", [0, 1])
def test_phase_graph_engine_matches_persistent(precision):
    """The graph of per-phase launches runs the persistent kernel's work units with
    the same operations and per-instance sums: bit-identical states and equal cycle
    and V-cycle counts after Step 0 and five steps, instances of uneven sizes
    (including the 96^2 and 128^2 ones of the sweep) and biases."""
    from paper_2210_15668_gb300 import ferrox
    rng = np.random.default_rng(21)
    sizes = [32, 128, 48, 96, 64, 32]
    geoms = [I.make_geometry(s, s, I.mfim_stack(16)) for s in sizes]
    P0s = [I.random_polarization(g, seed=200 + i) for i, g in enumerate(geoms)]
    biases = rng.uniform(-2.0, 2.0, size=len(geoms))
    num = ferrox.make_numerics(4e-13, tol=1e-10, precision=precision)
    outs = []
    for engine in (0, 1):
        B = ferrox.Batch(geoms, P0s, num)
        if engine == 0:
            B.set_shape(256, 1, 1, 0)
        else:
            B.set_engine(1)
        assert B.tuning()["engine"] == engine
        B.set_bias(np.zeros(len(geoms)), biases)
        B.solve_poisson()
        B.step(5)
        st = B.stats()
        assert all(x["status"] == 0 and x["steps"] == 5 for x in st)
        outs.append(([B.state(i) for i in range(len(geoms))],
                     [(x["cycles"], x["vcycles"], x["solves"]) for x in st]))
        B.close()
    (s0, c0), (s1, c1) = outs
    assert c1 == c0
    # both carry the full coarse-grid correction: the single-instance solver needs
    # 6-8 V-cycles per solve on these stacks, a V-cycle whose coarse levels
    # correct too little 18 or more
    assert all(c / s <= 10 for c, _, s in c0), c0
    for (P, phi), (Pr, phir) in zip(s1, s0):
        assert np.array_equal(P, Pr) and np.array_equal(phi, phir)


def test_set_engine_rejects_other_values():
    from paper_2210_15668_gb300 import ferrox
    geoms, P0s, _ = small_batch(n=2)
    B = ferrox.Batch(geoms, P0s, ferrox.make_numerics(4e-13))
    with pytest.raises(ferrox.FerroxError, match="EINVAL"):
        B.set_engine(2)
    B.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_phase_profile_advances_like_a_graph_step(precision):
    """ferrox_batch_profile_phases launches the graph engine's kernels one by one
    with the solve loop on the host: after it the state equals the state after one
    step of the graph, bit for bit, with equal counters, and every phase class the
    step runs has launches and time."""
    from paper_2210_15668_gb300 import ferrox
    sizes = [32, 96, 48]
    geoms = [I.make_geometry(s, s, I.mfim_stack(16)) for s in sizes]
    P0s = [I.random_polarization(g, seed=500 + i) for i, g in enumerate(geoms)]
    num = ferrox.make_numerics(4e-13, tol=1e-10, precision=precision)
    outs, prof = [], None
    for use_profile in (False, True):
        B = ferrox.Batch(geoms, P0s, num)
        B.set_engine(1)
        B.set_bias(np.zeros(len(sizes)), [-1.2, 0.4, 1.9])
        B.solve_poisson()
        if use_profile:
            prof = B.profile_phases()
        else:
            B.step(1)
        st = B.stats()
        outs.append(([B.state(i) for i in range(len(sizes))],
                     [(x["cycles"], x["vcycles"], x["solves"], x["steps"]) for x in st]))
        B.close()
    (s0, c0), (s1, c1) = outs
    assert c1 == c0 and all(c[3] == 1 for c in c0)
    for (P, phi), (Pr, phir) in zip(s1, s0):
        assert np.array_equal(P, Pr) and np.array_equal(phi, phir)
    assert prof["tdgl"][1] == 1
    assert prof["decide"][1] == prof["resid"][1] >= 2
    for k in ("tdgl", "resid", "decide", "smooth_fine", "transfer", "tail"):
        assert prof[k][1] > 0 and prof[k][0] > 0.0, (k, prof)


def test_phase_profile_needs_the_graph_engine():
    from paper_2210_15668_gb300 import ferrox
    geoms, P0s, _ = small_batch(n=2)
    B = ferrox.Batch(geoms, P0s, ferrox.make_numerics(4e-13))
    with pytest.raises(ferrox.FerroxError, match="ESTATE"):
        B.profile_phases()          # not tuned yet
    B.set_shape(256, 1, 1, 0)       # the persistent engine
    with pytest.raises(ferrox.FerroxError, match="ESTATE"):
        B.profile_phases()
    B.close()

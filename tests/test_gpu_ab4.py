"""GPU parity of the Adams-Bashforth push on the quartic path (FEMPIC_PUSH_AB4)
against the oracle, through the C ABI.

Every step starts both sides from the same fields (the oracle's e, b are set
on the device), so the particle half of each step is compared on its own
across the AB1 -> AB4 start-up.  The two sides find a face crossing
independently (the oracle from the roots of lambda_i(x(s)), the kernel by
Bernstein subdivision), so the decisions must agree exactly: owning tets,
crossing counts and crossing-sequence hashes bit-exact.  Velocities do not
depend on a crossing parameter (a wall mirrors them by its face alone):
bit-exact after the first step.  Positions depend on it only through wall
hit points: within 1e-12 of the unit box; those ~1e-16 differences feed the
next step's field gather, so later velocities are held to 1e-12 per
element.  The current per DOF within 1e-12 of the sum of the
absolute values of its terms (the crossing parameters agree to about 1e-12
in the worst-conditioned case and to rounding otherwise; atomics reorder the
sums), charge conserved on the device to 1e-12.
"""

import numpy as np
import pytest

import workloads
from oracle import sim as osim
from gpu_helpers import assert_close_to_scale, assert_elementwise, build_lib
from test_oracle_boundary_species import M_E, M_SR, Q_E

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    return build_lib()


def _setup(order, seed, species=False, n=1500):
    from paper_2111_12411_gb300 import Simulation
    xyz, tets = workloads.kuhn_box(4, 4, 4, jitter=0.1, seed=seed)
    rng = np.random.default_rng(seed)
    x, tet = workloads.sample_uniform_in_tets(xyz, tets, n, rng)
    # 0.05 m per step, gyroradius ~0.3 m (curved paths); omega_c dt = 0.18, inside the
    # Adams-Bashforth 4 stability interval on the imaginary axis (|omega dt| < ~0.43)
    v = workloads.maxwellian(n, 5e7, rng)
    sp = [dict(q=-Q_E, m=M_E, weight=1e4, x=x, v=v, tet=tet)]
    if species:
        xi, ti = workloads.sample_uniform_in_tets(xyz, tets, n // 3, rng)
        sp.append(dict(q=Q_E, m=M_SR, weight=1e4, x=xi, v=workloads.maxwellian(n // 3, 1e6, rng), tet=ti))
    o = osim.Sim(xyz, tets, order, -Q_E, M_E, 1e4, B0=(0.0, 0.0, 1e-3), push="ab4")
    o.set_species(sp)
    g = Simulation(xyz, tets, order, -Q_E, M_E, 1e4, x, v, tet, B0=(0.0, 0.0, 1e-3), es_init=False,
                   diagnostics=True, push="ab4", species=sp if species else None)
    t = o.topo
    o.e = workloads.random_dof_vector(t.n1, 3e3, rng, t.pec1)
    o.e_prev = o.e.copy()
    return o, g


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("species", [False, True])
def test_ab4_steps_match_oracle(order, species):
    o, g = _setup(order, 30 + order, species)
    dt = 1e-9
    for k in range(5):
        g.set("E", o.e)
        g.set("E_PREV", o.e_prev)
        g.set("B", o.b)
        w = o.step(dt)
        g.step(dt)
        assert w["order"] == min(4, k + 1)
        assert np.array_equal(g.get("TET"), w["tet"])
        assert np.array_equal(g.get("NCROSS"), w["ncross"])
        assert np.array_equal(g.get("HASH"), w["hash"])
        if k == 0:
            assert np.array_equal(g.get("V"), w["v"])
        assert_close_to_scale(g.get("V"), w["v"], 1e-12, "v")
        assert np.abs(g.get("X") - w["x"]).max() <= 1e-12
        assert_elementwise(g.get("DG"), w["dg"], w["dg_abs"], 1e-12, "dg")
        assert_elementwise(g.get("RHO"), o.rho, o.rho_abs, 1e-12, "rho")
        d = g.diag()
        assert d["continuity_abs"] <= 1e-12 * d["continuity_ref"]
    assert w["ncross"].sum() > 1000 and w["ncross"].max() < 50
    g.close()


def test_ab4_restarts_history_on_set():
    """Setting the particle state restarts the Adams-Bashforth order at 1, as
    a fresh oracle from the same state does."""
    o, g = _setup(1, 40, n=600)
    dt = 1e-9
    for _ in range(3):
        g.set("E", o.e)
        g.set("E_PREV", o.e_prev)
        g.set("B", o.b)
        o.step(dt)
        g.step(dt)
    x, v, tet = g.get("X"), g.get("V"), g.get("TET")
    g.set("X", x)
    g.set("V", v)
    g.set("TET", tet)
    fresh = osim.Sim(o.topo.xyz, o.topo.tets, 1, -Q_E, M_E, 1e4, B0=(0.0, 0.0, 1e-3), push="ab4")
    fresh.set_particles(x, v, tet)
    fresh.e, fresh.e_prev, fresh.b = o.e.copy(), o.e_prev.copy(), o.b.copy()
    g.set("E", fresh.e)
    g.set("E_PREV", fresh.e_prev)
    g.set("B", fresh.b)
    w = fresh.step(dt)
    g.step(dt)
    assert w["order"] == 1
    assert np.abs(g.get("X") - w["x"]).max() <= 1e-12 and np.array_equal(g.get("TET"), w["tet"])
    g.close()


def test_ab4_finds_a_crossing_pair_inside_one_eighth_of_the_step():
    """A path that leaves its tet through a face and comes back within one
    eighth of the step (the kind of excursion an eight-sample search misses):
    one electron in a uniform E field on an unjittered Kuhn box, started so
    that its second step (Adams-Bashforth 2) is the parabola
    z(s) = 0.5 + beta (s - 0.3)(s - 0.34) across the plane z = 0.5.  Device and
    oracle both count two crossings, end in the starting tet and agree on the
    crossing hash."""
    from paper_2111_12411_gb300 import Simulation
    from oracle import geometry, topology
    xyz, tets = workloads.kuhn_box(4, 4, 4)
    t = topology.Topology(xyz, tets, 1)
    g_all, c_all, _ = geometry.barycentric_maps(t.xyz, t.tets)
    dt, beta = 1e-9, 0.0375
    a_z = 2.0 * beta / dt ** 2
    v1 = np.array([0.0, 0.0, -0.64 * beta / dt])
    v0 = v1 - np.array([0.0, 0.0, dt * a_z])
    x1 = np.array([0.35, 0.30, 0.5 + 0.102 * beta])
    x0 = x1 - dt * v0
    E = np.array([0.0, 0.0, a_z * M_E / -Q_E])                 # electron: a = -(e/m) E
    e_dof = (t.xyz[t.edges[:, 1]] - t.xyz[t.edges[:, 0]]) @ E  # Whitney DOFs of the uniform field
    zs = [0.5 + beta * (s - 0.3) * (s - 0.34) for s in np.arange(9) / 8.0]
    assert min(zs) > 0.5                                        # every eighth of the step is above the plane
    lam = np.einsum("tik,k->ti", g_all, x0) + c_all
    tet0 = np.array([int(np.argmax(lam.min(axis=1)))])
    o = osim.Sim(xyz, tets, 1, -Q_E, M_E, 1.0, push="ab4")
    o.set_particles(x0[None], v0[None], tet0)
    g = Simulation(xyz, tets, 1, -Q_E, M_E, 1.0, x0[None], v0[None], tet0, push="ab4", es_init=False)
    for k in range(2):
        tet1 = int(o.tet[0])                                    # the tet the step starts in
        o.e, o.e_prev, o.b = e_dof.copy(), e_dof.copy(), np.zeros(t.n2)
        g.set("E", o.e)
        g.set("E_PREV", o.e_prev)
        g.set("B", o.b)
        w = o.step(dt)
        g.step(dt)
    assert w["order"] == 2
    assert w["ncross"][0] == 2 and w["tet"][0] == tet1          # out through z = 0.5 and back
    assert np.array_equal(g.get("NCROSS"), w["ncross"])
    assert np.array_equal(g.get("TET"), w["tet"])
    assert np.array_equal(g.get("HASH"), w["hash"])
    assert np.abs(g.get("X")[0] - w["x"][0]).max() <= 1e-12
    g.close()

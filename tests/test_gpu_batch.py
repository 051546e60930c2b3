"""GPU tests of batched execution: uneven instances (orders 1 and 2, FP64 and
mixed precision, different meshes and particle counts) advanced together in
one launch per kernel give, member by member, the same state as each instance
advanced alone.  Tolerances: positions/velocities rel 1e-9 after 3 steps in
FP64 (same arithmetic; only the order of the FP64 atomic current sums
differs, and it feeds the field solve), 2e-6 with the FP32 push (a last-bit
field difference can flip an FP32 rounding); fields rel 1e-6 (CG stopped at
rel 1e-12 residual on systems with condition numbers up to ~1e6); charge
conservation 1e-12.  After one step from the same field state the batched
particle kernel (the single-instance kernel's step, run per member) must give
bit-identical positions, velocities, tets and crossing hashes; and one batched
step of each member is checked against the oracle."""

import numpy as np
import pytest

import workloads
from oracle import fields as ofields, geometry, sim as osim, topology as otopo
from gpu_helpers import (assert_elementwise, assert_particles_close, assert_rho, assert_solves_system,
                         build_lib, random_state, rel)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    return build_lib()


def _instances():
    cfgs = workloads.make_batch(n_instances=5, np_range=(3e3, 3e4), nt_range=(2e3, 9e3), steps=3)
    cfgs[0]["precision"] = "fp64"
    cfgs[1]["precision"] = "mixed"
    return cfgs


def test_batch_matches_members_alone():
    from paper_2111_12411_gb300 import Batch, Simulation
    cfgs = _instances()
    assert len({c["order"] for c in cfgs}) == 2  # both orders in the mix
    alone = [Simulation.from_config(c) for c in cfgs]
    mixed = [Simulation.from_config(c) for c in cfgs]
    rng = np.random.default_rng(21)
    for a, m, c in zip(alone, mixed, cfgs):      # one field state for both (a kick of about v_th per step)
        e, b = random_state(otopo.Topology(c["xyz"], c["tets"], c["order"]), rng, e_scale=10.0, b_scale=1e-5)
        for s in (a, m):
            s.set("E", e)
            s.set("E_PREV", e)
            s.set("B", b)
    batch = Batch(mixed)
    dts = np.array([c["dt"] for c in cfgs])
    for s, c in zip(alone, cfgs):
        s.step(c["dt"])
    batch.step(dts)
    for k, (a, m) in enumerate(zip(alone, mixed)):
        for q in ("X", "V", "TET", "HASH", "NCROSS"):
            assert np.array_equal(m.get(q), a.get(q)), (k, q)
    for s, c in zip(alone, cfgs):
        s.step(c["dt"], 2)
    batch.step(dts, 2)
    t = batch.timing()
    assert t["launches_per_step"] > 0
    for k, (a, m, c) in enumerate(zip(alone, mixed, cfgs)):
        tol = 2e-6 if c["precision"] == "mixed" else 1e-9
        xa, xm = a.get("X"), m.get("X")
        assert rel(xm, xa) < tol, k
        assert rel(m.get("V"), a.get("V")) < tol, k
        assert (m.get("TET") == a.get("TET")).mean() > 0.999
        assert rel(m.get("E"), a.get("E")) < 1e-6, k
        assert rel(m.get("B"), a.get("B")) < 1e-6, k
    batch.close()
    for s in alone + mixed:
        s.close()


def test_batch_conserves_charge_per_member():
    from paper_2111_12411_gb300 import Batch, Simulation
    cfgs = _instances()[:3]
    sims = [Simulation.from_config(c) for c in cfgs]
    batch = Batch(sims)
    dts = np.array([c["dt"] for c in cfgs])
    batch.step(dts, 2)
    before = [s.get("RHO") for s in sims]
    batch.step(dts, 1)
    for s, c, r0 in zip(sims, cfgs, before):
        topo = otopo.Topology(c["xyz"], c["tets"], c["order"])
        drho = s.get("RHO") - r0
        res = drho - s.apply("DT", s.get("DG"))
        ii = topo.interior0
        assert np.linalg.norm(res[ii]) <= 1e-12 * np.linalg.norm(drho[ii])
    batch.close()
    for s in sims:
        s.close()


def test_autotune_picks_a_candidate_and_keeps_results():
    """The autotuner advances the members by real steps under each launch
    shape; afterwards the batch (now replaying a graph of the chosen shapes)
    still gives each member's state alone, to the tolerances above."""
    from paper_2111_12411_gb300 import Batch, Simulation
    cfgs = _instances()[:4]
    alone = [Simulation.from_config(c) for c in cfgs]
    mixed = [Simulation.from_config(c) for c in cfgs]
    batch = Batch(mixed)
    dts = np.array([c["dt"] for c in cfgs])
    t = batch.autotune(dts, steps_per_candidate=1)
    assert t["particle_block"] in (128, 256) and t["particle_grid"] > 0
    assert 1 <= t["cg_ctas_per_sm"] and t["particle_candidates"] >= 3 and t["cg_candidates"] >= 1
    assert t["steps"] == max(t["particle_candidates"], t["cg_candidates"])
    assert 0 < t["particle_ms"] <= t["particle_ms_default"] and 0 < t["cg_ms"] <= t["cg_ms_default"]
    batch.step(dts, 2)
    assert batch.timing()["graph"] == 1.0
    for s, c in zip(alone, cfgs):
        s.step(c["dt"], t["steps"] + 2)
    for k, (a, m, c) in enumerate(zip(alone, mixed, cfgs)):
        tol = 2e-6 if c["precision"] == "mixed" else 1e-9
        assert rel(m.get("X"), a.get("X")) < tol, k
        assert rel(m.get("V"), a.get("V")) < tol, k
        assert rel(m.get("E"), a.get("E")) < 1e-6, k
    batch.close()
    for s in alone + mixed:
        s.close()


def test_batch_member_one_step_matches_oracle():
    """One batched step (Section III-B cycle) of an order-1 and an order-2 FP64
    member and an order-2 mixed member, each from a random field state set on
    both sides, against the oracle.  FP64 (contracted) members: positions
    within 1e-12 of the unit box, velocities within 1e-12 of each particle's
    speed, tets, crossing counts and hashes equal, the current per DOF within
    1e-11 of its terms (midpoint against 2-point Gauss rule), the charge at the
    member's own end points, the field solve satisfying the oracle's system,
    b^{n+1} equal to the oracle's Faraday update of the member's own e^{n+1}.
    Mixed member (FP32 gather and push): positions within 2e-6 of the box,
    velocities within 2e-6 of the speed, tets equal where the end point is
    not within 1e-5 of a face.  Charge conserved on the device for every
    member."""
    from paper_2111_12411_gb300 import Batch, Simulation
    cfgs = workloads.make_batch(n_instances=3, np_range=(4e3, 8e3), nt_range=(2e3, 4e3), steps=1,
                                seed=77, precision="fp64")
    cfgs[0]["order"], cfgs[1]["order"], cfgs[2]["order"] = 1, 2, 2
    cfgs[2]["precision"] = "mixed"
    rng = np.random.default_rng(22)
    sims, oracles = [], []
    for c in cfgs:
        o = osim.Sim(c["xyz"], c["tets"], c["order"], c["q"], c["m"], c["weight"], c["B0"], c["rho_ion"])
        o.set_particles(c["x"], c["v"], c["tet"])
        e, b = random_state(o.topo, rng, e_scale=10.0, b_scale=1e-5)
        o.e, o.e_prev, o.b = e.copy(), e.copy(), b.copy()
        g = Simulation.from_config(c, es_init=False, diagnostics=True)
        g.set("E", e)
        g.set("E_PREV", e)
        g.set("B", b)
        sims.append(g)
        oracles.append((o, e, b))
    batch = Batch(sims)
    batch.step(np.array([c["dt"] for c in cfgs]))
    for k, (g, (o, e, b), c) in enumerate(zip(sims, oracles, cfgs)):
        w = o.step(c["dt"])
        d = g.diag()
        assert d["continuity_abs"] <= 1e-12 * d["continuity_ref"], k
        if c["precision"] == "mixed":
            assert_particles_close(g.get("X"), g.get("V"), w["x"], w["v"], 2e-6, 1.0, f"[{k}]")
            ok = geometry.lam(o.g[w["tet"]], o.c[w["tet"]], w["x"]).min(axis=1) > 1e-5
            assert ok.mean() > 0.98
            assert np.array_equal(g.get("TET")[ok], w["tet"][ok]), k
            continue
        assert_particles_close(g.get("X"), g.get("V"), w["x"], w["v"], 1e-12, 1.0, f"[{k}]")  # unit box
        for q, key in (("TET", "tet"), ("NCROSS", "ncross"), ("HASH", "hash")):
            assert np.array_equal(g.get(q), w[key]), (k, q)
        assert_elementwise(g.get("DG"), w["dg"], w["dg_abs"], 1e-11, f"dg[{k}]")
        assert_rho(g.get("RHO"), o, "fp64", f"rho[{k}]", g.get("X"), g.get("TET"))
        A = ofields.system_matrix(o.M, o.K, c["dt"], "trapezoid")
        eg = g.get("E")
        fr = o.topo.free1
        dgg = g.get("DG")                    # the member's own current, as on the device
        rhs = ofields.rhs_trapezoid(o.M, o.K, o.CtM2, e, b, dgg, c["dt"])
        terms = abs(o.M) @ np.abs(e) + (0.25 * c["dt"] ** 2) * (abs(o.K) @ np.abs(e)) \
            + c["dt"] * (abs(o.CtM2) @ np.abs(b)) + np.abs(dgg)
        assert_solves_system(A[fr][:, fr], eg[fr], rhs[fr], terms[fr], 1e-12, f"e[{k}]")
        want = ofields.update_b(o.C, b, eg, e, c["dt"])
        scale = np.abs(b) + (0.5 * c["dt"]) * (abs(o.C) @ (np.abs(eg) + np.abs(e)))
        assert_elementwise(g.get("B"), want, scale, 1e-13, f"b[{k}]")
    batch.close()
    for g in sims:
        g.close()

"""GPU tests of batched execution: uneven instances (orders 1 and 2, FP64 and
mixed precision, different meshes and particle counts) advanced together in
one launch per kernel give, member by member, the same state as each instance
advanced alone.  Tolerances: positions/velocities rel 1e-9 after 3 steps in
FP64 (same arithmetic; only the order of the FP64 atomic current sums
differs, and it feeds the field solve), 2e-6 with the FP32 push (a last-bit
field difference can flip an FP32 rounding); fields rel 1e-6 (CG stopped at
rel 1e-12 residual on systems with condition numbers up to ~1e6); charge
conservation 1e-12."""

import numpy as np
import pytest

import workloads
from oracle import topology as otopo
from gpu_helpers import build_lib, rel

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
    batch = Batch(mixed)
    dts = np.array([c["dt"] for c in cfgs])
    rho0 = [s.get("RHO") for s in mixed]
    for s, c in zip(alone, cfgs):
        s.step(c["dt"], 3)
    batch.step(dts, 3)
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

"""GPU test of the serving loop: requests of different meshes, orders and
particle counts arrive over time, are admitted under an HBM budget that does
not hold them all at once, advance in chunks together with whatever else is
resident (continuous batching), and each result equals the same request
simulated alone (positions rel 1e-9 in FP64, 2e-6 with the FP32 push; fields
rel 1e-6, as in the batch test)."""

import numpy as np
import pytest

import workloads
from gpu_helpers import build_lib, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    return build_lib()


def test_serving_continuous_batching_results_match_alone():
    from paper_2111_12411_gb300 import Simulation
    from paper_2111_12411_gb300.serve import Request, Server

    rng = np.random.default_rng(9)
    reqs = []
    for i in range(6):
        n = int(rng.integers(6, 10))
        cfg = workloads.configs._box_instance(n, int(rng.integers(1, 3)), int(rng.integers(2000, 20000)),
                                              1.0e6, float(rng.uniform(0, 1)), 1000 + i,
                                              precision="mixed" if i % 2 else "fp64", steps=6)
        reqs.append(Request(i, cfg, arrival=0.05 * i, n_chunks=int(rng.integers(1, 4)), chunk_steps=3))
    budget = sum(sorted(r.bytes for r in reqs)[-3:])  # at most ~3 resident at a time
    server = Server(budget, max_slots=4, result_keys=("X", "E", "RHO"))
    for r in reqs:
        server.submit(r)
    done = server.run(max_wall_s=600)
    assert len(done) == len(reqs)
    rep = server.report()
    assert rep["p50_chunk_latency_s"] > 0 and rep["p99_chunk_latency_s"] >= rep["p50_chunk_latency_s"]
    # admission happened while others were still running
    overlap = any(a.admitted_at < b.finished_at and a.admitted_at > b.admitted_at
                  for a in done for b in done if a is not b)
    assert overlap
    assert max(len([r for r in done if r.admitted_at <= t < r.finished_at])
               for t in [r.admitted_at for r in done]) >= 2
    for r in done:
        alone = Simulation.from_config(r.cfg)
        alone.step(r.cfg["dt"], r.n_chunks * r.chunk_steps)
        tol = 2e-6 if r.cfg["precision"] == "mixed" else 1e-9
        assert rel(r.result["X"], alone.get("X")) < tol, r.id
        assert rel(r.result["E"], alone.get("E")) < 1e-6, r.id
        assert rel(r.result["RHO"], alone.get("RHO")) < tol, r.id
        alone.close()


def test_served_requests_match_oracle():
    """Four requests (orders 1 and 2, FP64 and FP32 push) admitted together
    and advanced in one batch by one step each; each result is checked
    against the oracle's step (Section III-B cycle) of the request's own inputs
    from the device's electrostatic start e^0 (read back as E_PREV).  FP64:
    positions within 1e-12 of the unit box, velocities within 1e-12 of each
    particle's speed, tets,
    crossing counts and hashes equal, current per DOF within 1e-11 of its
    terms; FP32 push: positions within 2e-6 of the box and velocities within
    2e-6 of the speed, tets equal where
    the end point is not within 1e-5 of a face.  Every request's e^{n+1}
    satisfies the oracle's trapezoidal system built from its own e^0 and
    Delta g to 10 cg_rtol plus the rounding of the right-hand side's terms."""
    from oracle import fields as ofields, geometry, sim as osim
    from paper_2111_12411_gb300.serve import Request, Server
    from gpu_helpers import assert_elementwise, assert_particles_close, assert_rho, assert_solves_system

    reqs = []
    for i, (order, prec) in enumerate([(1, "fp64"), (2, "fp64"), (1, "mixed"), (2, "mixed")]):
        cfg = workloads.configs._box_instance(6, order, 3000 + 500 * i, 1.0e6, 0.3, 2000 + i,
                                              precision=prec, steps=1)
        reqs.append(Request(i, cfg, arrival=0.0, n_chunks=1, chunk_steps=1))
    server = Server(sum(r.bytes for r in reqs), max_slots=4,
                    result_keys=("X", "V", "TET", "NCROSS", "HASH", "E", "E_PREV", "DG", "RHO"))
    for r in reqs:
        server.submit(r)
    done = server.run(max_wall_s=600)
    assert len(done) == len(reqs)
    for r in done:
        c, res = r.cfg, r.result
        o = osim.Sim(c["xyz"], c["tets"], c["order"], c["q"], c["m"], c["weight"], c["B0"], c["rho_ion"])
        o.set_particles(c["x"], c["v"], c["tet"])
        e0 = res["E_PREV"]
        o.e, o.e_prev = e0.copy(), e0.copy()
        w = o.step(c["dt"])
        if c["precision"] == "mixed":
            assert_particles_close(res["X"], res["V"], w["x"], w["v"], 2e-6, 1.0, f"[{r.id}]")
            ok = geometry.lam(o.g[w["tet"]], o.c[w["tet"]], w["x"]).min(axis=1) > 1e-5
            assert ok.mean() > 0.98
            assert np.array_equal(res["TET"][ok], w["tet"][ok]), r.id
        else:
            assert_particles_close(res["X"], res["V"], w["x"], w["v"], 1e-12, 1.0, f"[{r.id}]")  # unit box
            assert np.array_equal(res["TET"], w["tet"]), r.id
            assert np.array_equal(res["NCROSS"], w["ncross"]), r.id
            assert np.array_equal(res["HASH"], w["hash"]), r.id
            assert_elementwise(res["DG"], w["dg"], w["dg_abs"], 1e-11, f"dg[{r.id}]")
            assert_rho(res["RHO"], o, "fp64", f"rho[{r.id}]", res["X"], res["TET"])
        A = ofields.system_matrix(o.M, o.K, c["dt"], "trapezoid")
        rhs = ofields.rhs_trapezoid(o.M, o.K, o.CtM2, e0, np.zeros(o.topo.n2), res["DG"], c["dt"])
        fr = o.topo.free1
        # e^0 is a gradient field, so M e^0 - dt^2/4 K e^0 cancels: the check allows the
        # rounding of those terms (assert_solves_system)
        terms = abs(o.M) @ np.abs(e0) + (0.25 * c["dt"] ** 2) * (abs(o.K) @ np.abs(e0)) + np.abs(res["DG"])
        assert_solves_system(A[fr][:, fr], res["E"][fr], rhs[fr], terms[fr], 1e-12, f"e[{r.id}]")

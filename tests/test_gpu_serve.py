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

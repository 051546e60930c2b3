"""GPU test of femPIC_eval_fields_noalloc, the field probe that makes no device
allocation (for callers that must not allocate device memory while they run,
such as a serving loop whose HBM budget is spoken for, or a latency-critical
loop that cannot take the device synchronisation cudaMalloc/cudaFree imply).

It must return exactly what femPIC_eval_fields returns (the same kernel on
the same inputs, staged through the library's fixed device array instead of
per-call buffers), on two calls in a row with different point sets, and refuse
more points than the array holds.  This file is collected last on purpose.
"""

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nat():
    from paper_2111_12411_gb300 import build
    build.build()
    from paper_2111_12411_gb300 import native
    native.load()
    return native


@pytest.mark.parametrize("order,precision", [(1, "fp64"), (2, "fp64_strict")])
def test_noalloc_probe_matches_eval_fields(nat, order, precision):
    from oracle import topology
    cfg = workloads.make_config(0, n_particles=20_000)
    sim = nat.Simulation(cfg["xyz"], cfg["tets"], order, cfg["q"], cfg["m"], cfg["weight"],
                         cfg["x"], cfg["v"], cfg["tet"], precision=precision, B0=cfg["B0"],
                         es_init=False)
    t = topology.Topology(cfg["xyz"], cfg["tets"], order)
    rng = np.random.default_rng(42)
    sim.set("E", workloads.random_dof_vector(t.n1, 1e3, rng, t.pec1))
    sim.set("B", workloads.random_dof_vector(t.n2, 1e-4, rng))
    # two calls in a row: different sizes and points; the second call reuses the
    # array that still holds the first call's data
    allocs = lambda: nat.femPIC_get_info(sim.h).device_allocations
    for lo, hi in ((0, 1_000), (3_000, 17_777)):
        x, tet = cfg["x"][lo:hi], cfg["tet"][lo:hi]
        a0 = allocs()
        E_ref, B_ref = nat.femPIC_eval_fields(sim.h, x, tet)
        a1 = allocs()
        E, B = nat.femPIC_eval_fields_noalloc(sim.h, x, tet)
        a2 = allocs()
        assert np.array_equal(E, E_ref) and np.array_equal(B, B_ref)
        assert np.abs(E).max() > 0 and np.abs(B).max() > 0
        # the library's device-allocation count: the allocating probe raises it,
        # this one leaves it where it was
        assert a1 > a0 and a2 == a1
    sim.close()


def test_noalloc_probe_rejects_too_many_points(nat):
    cfg = workloads.make_config(0, n_particles=100)
    sim = nat.Simulation.from_config(cfg, es_init=False)
    n = nat.FEMPIC_PROBE_MAX_POINTS + 1
    x = np.repeat(cfg["x"][:1], n, axis=0)
    tet = np.repeat(cfg["tet"][:1], n)
    with pytest.raises(nat.FemPICError) as ei:
        nat.femPIC_eval_fields_noalloc(sim.h, x, tet)
    assert ei.value.code == nat.FEMPIC_ERR_SIZE
    assert "FEMPIC_PROBE_MAX_POINTS" in str(ei.value)
    # the largest allowed call still works and matches
    E_ref, B_ref = nat.femPIC_eval_fields(sim.h, x[:-1], tet[:-1])
    E, B = nat.femPIC_eval_fields_noalloc(sim.h, x[:-1], tet[:-1])
    assert np.array_equal(E, E_ref) and np.array_equal(B, B_ref)
    sim.close()

"""GPU parity of the impedance (first-order absorbing) boundary and of several
species, through femPIC_create_ext, against the oracle.

Tolerances as in test_gpu_parity: strict FP64 particle state and walk
decisions bit-exact, Delta g and rho normwise rel 1e-12, the field solve
satisfies the oracle's system (which carries dt/2 [*_I] on both sides for
impedance faces) to 10 cg_rtol.  The energy balance of the trapezoid rule is
checked to the accuracy the CG tolerance allows.
"""

import numpy as np
import pytest

import workloads
from oracle import fields as ofields, sim as osim
from gpu_helpers import assert_elementwise, build_lib, rel, assert_rho
from test_oracle_boundary_species import M_E, M_SR, Q_E, tags_on_plane

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    return build_lib()


def _mesh():
    xyz, tets = workloads.kuhn_box(4, 4, 4, jitter=0.1, seed=21)
    rng = np.random.default_rng(3)
    perm = np.array([rng.permutation(4) for _ in range(len(tets))])
    tets = np.take_along_axis(np.asarray(tets), perm, axis=1)  # vertex order as given, unsorted
    tag = tags_on_plane(xyz, tets, 0, 1.0) | tags_on_plane(xyz, tets, 2, 0.0)
    return xyz, tets, tag


def _species(xyz, tets, rng, n_e=3001, n_i=1499):
    xe, te = workloads.sample_uniform_in_tets(xyz, tets, n_e, rng)
    xi, ti = workloads.sample_uniform_in_tets(xyz, tets, n_i, rng)
    return [dict(q=-Q_E, m=M_E, weight=2e5, x=xe, v=workloads.maxwellian(n_e, 2e6, rng), tet=te),
            dict(q=Q_E, m=M_SR, weight=3e5, x=xi, v=workloads.maxwellian(n_i, 5e4, rng), tet=ti)]


@pytest.mark.parametrize("order", [1, 2, 3])
@pytest.mark.parametrize("precision", ["fp64_strict", "fp64", "mixed"])
def test_ions_electrons_and_impedance_step(order, precision):
    from paper_2111_12411_gb300 import Simulation
    xyz, tets, tag = _mesh()
    rng = np.random.default_rng(8)
    sp = _species(xyz, tets, rng)
    o = osim.Sim(xyz, tets, order, -Q_E, M_E, 2e5, B0=(0.0, 0.0, 0.05), bface_tag=tag)
    o.set_species(sp)
    g = Simulation(xyz, tets, order, -Q_E, M_E, 2e5, sp[0]["x"], sp[0]["v"], sp[0]["tet"],
                   precision=precision, B0=(0.0, 0.0, 0.05), es_init=False, diagnostics=True,
                   species=sp, bface_tag=tag)
    t = o.topo
    assert g.info.n_species == 2 and g.info.n_impedance_faces == int(t.imp_face.sum()) > 0
    assert np.array_equal(g.get("SPECIES"), np.repeat([0, 1], [3001, 1499]))
    assert_rho(g.get("RHO"), o, precision, "rho at create")
    e = workloads.random_dof_vector(t.n1, 1e3, rng, t.pec1)
    b = workloads.random_dof_vector(t.n2, 1e-4, rng)
    o.e, o.e_prev, o.b = e.copy(), e.copy(), b.copy()
    g.set("E", e)
    g.set("E_PREV", e)
    g.set("B", b)
    dt = 2e-10
    w = o.step(dt)
    g.step(dt)
    xg, vg, tg = g.get("X"), g.get("V"), g.get("TET")
    if precision == "fp64_strict":
        assert np.array_equal(xg, w["x"]) and np.array_equal(vg, w["v"])
        assert np.array_equal(tg, w["tet"])
        assert np.array_equal(g.get("HASH"), w["hash"])
    else:
        tol = 1e-12 if precision == "fp64" else 2e-6
        assert rel(xg, w["x"]) < tol and rel(vg, w["v"]) < tol
    dg = g.get("DG")
    if precision != "mixed":
        assert_elementwise(dg, w["dg"], w["dg_abs"], 1e-12 if precision == "fp64_strict" else 1e-11, "dg")
        assert_rho(g.get("RHO"), o, precision, "rho", g.get("X"), g.get("TET"))
    d = g.diag()
    assert d["continuity_abs"] <= 1e-12 * d["continuity_ref"]
    # the GPU's e^{n+1} solves the oracle's impedance system for the GPU's own current
    A = ofields.system_matrix(o.M, o.K, dt, "trapezoid", I=o.I)
    rhs = ofields.rhs_trapezoid(o.M, o.K, o.CtM2, e, b, dg, dt, o.I)
    eg = g.get("E")
    fr = t.free1
    res = (A @ eg - rhs)[fr]
    assert np.linalg.norm(res) <= 10 * 1e-12 * np.linalg.norm(rhs[fr])
    assert np.all(eg[~fr] == 0.0)
    if precision != "mixed":
        assert rel(eg, o.e) < 1e-6 and rel(g.get("B"), o.b) < 1e-6
    g.close()


@pytest.mark.parametrize("order", [1, 2])
def test_impedance_energy_balance_on_gpu(order):
    """Source-free fields through the absorbing faces: each step loses
    dt ebar.[*_I] ebar of e.[*eps]e/2 + b.[*mu^-1]b/2 (the oracle's matrices
    measure the GPU's fields)."""
    from paper_2111_12411_gb300 import Simulation
    xyz, tets, tag = _mesh()
    rng = np.random.default_rng(9)
    x, tt = workloads.sample_uniform_in_tets(xyz, tets, 33, rng)
    v = workloads.maxwellian(33, 1e5, rng)
    o = osim.Sim(xyz, tets, order, -Q_E, M_E, 0.0, bface_tag=tag)
    g = Simulation(xyz, tets, order, -Q_E, M_E, 0.0, x, v, tt, es_init=False, bface_tag=tag)
    t = o.topo
    e = workloads.random_dof_vector(t.n1, 1.0, rng, t.pec1)
    b = workloads.random_dof_vector(t.n2, 1e-8, rng)
    g.set("E", e)
    g.set("E_PREV", e)
    g.set("B", b)
    energy = lambda e_, b_: 0.5 * e_ @ (o.M @ e_) + 0.5 * b_ @ (o.M2 @ b_)
    dt = 2e-10
    for _ in range(3):
        e0, b0 = g.get("E"), g.get("B")
        g.step(dt)
        e1, b1 = g.get("E"), g.get("B")
        eb = 0.5 * (e0 + e1)
        loss = dt * eb @ (o.I @ eb)
        w0 = energy(e0, b0)
        assert loss > 1e-6 * w0
        assert abs((w0 - energy(e1, b1)) - loss) <= 1e-6 * loss + 1e-10 * w0
    g.close()


def test_several_species_cannot_join_a_batch():
    from paper_2111_12411_gb300 import Batch, FemPICError, Simulation
    xyz, tets, tag = _mesh()
    rng = np.random.default_rng(10)
    sp = _species(xyz, tets, rng, 64, 32)
    g = Simulation(xyz, tets, 1, -Q_E, M_E, 2e5, sp[0]["x"], sp[0]["v"], sp[0]["tet"], es_init=False,
                   species=sp)
    with pytest.raises(FemPICError):
        Batch([g])
    g.close()

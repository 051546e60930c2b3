"""GPU parity of the divergence-free projection of an impressed flux density
(Section III-C, eq. conB) against the oracle, through the C ABI.

* quadrature points: the library's rule equals the oracle's conical-product
  rule (p + 3 Gauss-Legendre points per direction), points to 1e-14;
* coefficients: the oracle solves the saddle-point system directly, the
  library by nested CG (inner rtol 1e-14, outer 1e-12): rel 1e-9;
* Gauss's magnetic law: ||div b|| / ||B|| <= 1e-11 with the constraint, as in
  the oracle, and the Galerkin projection is not divergence free;
* the particles sample B0 + (b + b_impressed) . W2, the field update b alone.
"""

import numpy as np
import pytest

import workloads
from oracle import geometry, particles as opart, project, topology
from gpu_helpers import build_lib, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    return build_lib()


def _sin(x):
    return np.stack([np.sin(x[:, 1]), np.cos(x[:, 0]), 0 * x[:, 0]], axis=1)


def _quad(x):
    """A quadrupole-like static field, divergence- and curl-free (the gradient
    of xy (1 + 0.3 z)), in tesla."""
    return np.stack([x[:, 1] * (1 + 0.3 * x[:, 2]), x[:, 0] * (1 + 0.3 * x[:, 2]), 0.3 * x[:, 0] * x[:, 1]],
                    axis=1) * 1e-2


def _setup(order, n=3, seed=3, np_=257):
    from paper_2111_12411_gb300 import Simulation
    xyz, tets = workloads.kuhn_box(n, n, n, lengths=(2.0, 2.0, 2.0), jitter=0.1, seed=seed)
    rng = np.random.default_rng(seed)
    x, tet = workloads.sample_uniform_in_tets(xyz, tets, np_, rng)
    v = workloads.maxwellian(np_, 1e6, rng)
    g = Simulation(xyz, tets, order, -1.602176634e-19, 9.1093837015e-31, 1.0, x, v, tet, B0=(0.0, 0.0, 0.0),
                   es_init=False, diagnostics=True)
    t = topology.Topology(xyz, tets, order)
    gg, c, vol = geometry.barycentric_maps(t.xyz, t.tets)
    return g, t, gg, c, vol, x, tet


@pytest.mark.parametrize("order", [1, 2, 3])
def test_points_match_the_rule(order):
    g, t, gg, c, vol, _, _ = _setup(order)
    pts = g.impressed_points()
    from oracle.quadrature import tet_rule
    lam, _ = tet_rule(order + 3)
    want = np.einsum("qk,tkd->tqd", lam, t.xyz[t.tets]).reshape(-1, 3)
    assert pts.shape == want.shape
    assert np.abs(pts - want).max() <= 1e-14 * np.abs(want).max()
    g.close()


@pytest.mark.parametrize("order", [1, 2, 3])
@pytest.mark.parametrize("field", ["sin", "quad"])
def test_projection_matches_oracle(order, field):
    f = {"sin": _sin, "quad": _quad}[field]
    g, t, gg, c, vol, _, _ = _setup(order)
    for constrained in (False, True):
        st = g.set_impressed_B(f, constrained=constrained)
        got = g.get("B_IMPRESSED")
        want = project.project(t, gg, vol, f, constrained=constrained)
        assert rel(got, want) < 1e-9, (constrained, rel(got, want), st)
        err, div = project.errors(t, gg, c, vol, got, f)
        err_o, div_o = project.errors(t, gg, c, vol, want, f)
        assert abs(err - err_o) <= 1e-6 * err_o + 1e-12  # the quadratic field is exact at order 3
        if constrained:
            assert div < 1e-11
        if field == "sin":  # not in the discrete space at any order: the Galerkin b is not div-free
            if constrained:
                assert st["div_residual"] < 1e-11 and st["outer_iterations"] > 0
            else:
                assert div > 1e4 * 1e-11
        assert st["inner_iterations"] > 0
    g.close()


@pytest.mark.parametrize("order", [1, 2, 3])
def test_particles_sample_the_impressed_field(order):
    g, t, gg, c, vol, x, tet = _setup(order)
    g.set_impressed_B(_quad, constrained=True)
    bi = g.get("B_IMPRESSED")
    rng = np.random.default_rng(7)
    b = workloads.random_dof_vector(t.n2, 1e-4, rng)
    g.set("B", b)
    assert np.array_equal(g.get("B"), b)                  # the self field is kept apart
    E, B = g.eval_fields(x, tet)
    _, Bo = opart.gather(t, gg, c, np.zeros(t.n1), b + bi, (0.0, 0.0, 0.0), x, tet)
    assert rel(B, Bo) < 1e-13
    # a step (moves of ~0.05 m in cells of ~0.7 m) keeps the impressed part
    # out of the field update and conserves charge
    g.step(5e-8)
    d = g.diag()
    assert d["continuity_abs"] <= 1e-12 * d["continuity_ref"]
    assert np.array_equal(g.get("B_IMPRESSED"), bi)
    _, B1 = g.eval_fields(x, tet)
    _, B1o = opart.gather(t, gg, c, np.zeros(t.n1), g.get("B") + bi, (0.0, 0.0, 0.0), x, tet)
    assert rel(B1, B1o) < 1e-13
    # clearing it: back to the self field
    g.set_impressed_B(None)
    assert not np.any(g.get("B_IMPRESSED"))
    _, B2 = g.eval_fields(x, tet)
    _, B2o = opart.gather(t, gg, c, np.zeros(t.n1), g.get("B"), (0.0, 0.0, 0.0), x, tet)
    assert rel(B2, B2o) < 1e-13
    g.close()


def test_projection_errors_and_batch_rejection():
    from paper_2111_12411_gb300 import Batch, FemPICError, native
    g, t, gg, c, vol, _, _ = _setup(2)
    with pytest.raises(FemPICError) as ei:
        native.femPIC_set_impressed_B(g.h, np.zeros((5, 3)))
    assert ei.value.code == native.FEMPIC_ERR_SIZE
    g.set("B_IMPRESSED", np.full(t.n2, 1e-3))              # coefficients set directly
    with pytest.raises(FemPICError):
        Batch([g])
    g.close()


@pytest.mark.parametrize("order", [1, 2, 3])
def test_divb_diagnostic(order):
    """The library's Gauss's-magnetic-law diagnostic equals ||[~div] b|| of
    the oracle's operator (rel 1e-12), and a divergence-free b stays so under
    the Faraday update (the curl map's range is divergence free)."""
    g, t, gg, c, vol, x, tet = _setup(order)
    S3, Dv, M2 = project.matrices(t, gg, vol)
    b = workloads.random_dof_vector(t.n2, 1e-4, np.random.default_rng(11))
    g.set("B", b)
    g.step(5e-8)
    d = g.diag()
    want = np.linalg.norm(Dv @ g.get("B"))
    assert abs(d["divb_abs"] - want) <= 1e-12 * want
    assert d["divb_ref"] >= d["divb_abs"]
    bf = project.project(t, gg, vol, _quad, constrained=True)
    g.set("B", bf)
    g.step(5e-8)
    d = g.diag()
    assert d["divb_ref"] > 0 and d["divb_abs"] <= 1e-12 * d["divb_ref"]
    g.close()

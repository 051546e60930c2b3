"""GPU parity of the walk on degenerate chords (Section III-B: the path is cut
into one sub-path per tet by intersecting it with the faces).  The tie-break
reading: exit candidates are the faces with lambda_i(b) < 0 other than the
entry face, the smallest crossing parameter wins, ties go to the lowest local
face, a tet is closed (lambda = 0 stays inside).

Chords through mesh vertices, through points of edges (axis, face-diagonal
and cell-diagonal edges of the Kuhn split), starting on a face, ending on a
face, lying in a face and starting at a vertex:
* on an unjittered Kuhn box with dyadic coordinates, where lambda is exactly
  zero at those points, so every tie is a real tie;
* on the unjittered drift-tube mesh (polar grid), where the same chords are
  degenerate up to rounding.
With no field the push leaves the velocity unchanged, so the chord is exactly
the one built here.  Strict FP64 mode: owning tets, crossing counts,
crossing-sequence hashes, positions and velocities bit-exact against the
oracle; the current per DOF within 1e-12 of the sum of the absolute values of
its terms, charge conserved on the device.
"""

import numpy as np
import pytest

import workloads
from oracle import geometry, sim as osim, topology as otopo
from gpu_helpers import assert_elementwise, build_lib

pytestmark = pytest.mark.gpu

Q_E = 1.602176634e-19
M_E = 9.1093837015e-31


@pytest.fixture(scope="module", autouse=True)
def lib():
    return build_lib()


def _owner(g, c, x):
    lam = np.einsum("tik,pk->pti", g, x) + c[None]
    return np.argmax(lam.min(axis=2), axis=1)


def degenerate_chords(xyz, tets, rng, n_each, scale, dyadic):
    """(x0, x1) pairs through special points of the mesh; ``scale`` is the
    chord half-length, ``dyadic`` rounds directions to multiples of scale/8."""
    t = otopo.Topology(xyz, tets, 1)
    lo, hi = xyz.min(axis=0), xyz.max(axis=0)

    def direction(k):
        d = rng.standard_normal((k, 3))
        d *= scale / np.linalg.norm(d, axis=1)[:, None]
        if dyadic:
            d = np.round(d * (8.0 / scale)) * (scale / 8.0)
            d[np.all(d == 0.0, axis=1)] = scale / 8.0
        return d

    def pick(a, k):
        return a[rng.integers(0, len(a), k)]

    verts = t.xyz
    edges = 0.5 * (t.xyz[t.edges[:, 0]] + t.xyz[t.edges[:, 1]])
    fv = t.xyz[t.faces]                                             # [F, 3, 3]
    wts = np.array([[0.5, 0.25, 0.25], [0.25, 0.5, 0.25], [0.25, 0.25, 0.5]])
    face_pts = np.einsum("wk,fkd->fwd", wts, fv)                     # [F, 3, 3]
    fsel = rng.integers(0, len(fv), n_each)
    fp = face_pts[fsel, 0]
    fq = face_pts[fsel, 1]
    x0, x1 = [], []
    for P in (pick(verts, n_each), pick(edges, n_each)):             # through vertex / edge points
        d = direction(n_each)
        x0.append(P - d)
        x1.append(P + d)
    d = direction(n_each)
    x0.append(fp)                                                    # starts on a face
    x1.append(fp + d)
    d = direction(n_each)
    x0.append(fp - d)                                                # ends on a face
    x1.append(fp)
    x0.append(fp)                                                    # lies in a face
    x1.append(fq)
    P = pick(verts, n_each)                                          # starts at a vertex
    x0.append(P)
    x1.append(P + direction(n_each))
    x0, x1 = np.concatenate(x0), np.concatenate(x1)
    inside = np.all((x0 >= lo) & (x0 <= hi) & (x1 >= lo) & (x1 <= hi), axis=1)
    return x0[inside], x1[inside]


def _run(xyz, tets, order, x0, x1, dt):
    t = otopo.Topology(xyz, tets, 1)
    g_all, c_all, _ = geometry.barycentric_maps(t.xyz, t.tets)
    tet = _owner(g_all, c_all, x0)
    inside = geometry.lam(g_all[tet], c_all[tet], x0).min(axis=1) >= -1e-12   # starts in the mesh
    x0, x1, tet = x0[inside], x1[inside], tet[inside]
    v = (x1 - x0) / dt
    w_part = 1.0
    o = osim.Sim(xyz, tets, order, -Q_E, M_E, w_part)
    o.set_particles(x0, v, tet)
    from paper_2111_12411_gb300 import Simulation
    g = Simulation(xyz, tets, order, -Q_E, M_E, w_part, x0, v, tet, precision="fp64_strict",
                   es_init=False, diagnostics=True)
    w = o.step(dt)
    g.step(dt)
    return o, g, w


@pytest.mark.parametrize("order", [1, 2])
def test_degenerate_chords_kuhn_box(order):
    xyz, tets = workloads.kuhn_box(4, 4, 4)
    rng = np.random.default_rng(70 + order)
    x0, x1 = degenerate_chords(xyz, tets, rng, 300, 0.25, dyadic=True)
    dt = 2.0 ** -30                       # exact: x0 + dt (x1 - x0) / dt == x1
    o, g, w = _run(xyz, tets, order, x0, x1, dt)
    assert len(w["x"]) == len(x1)
    assert np.array_equal(w["x"], x1)     # the box is convex: no chord meets a wall
    _compare(o, g, w)


@pytest.mark.parametrize("order", [1, 2])
def test_degenerate_chords_drift_tube(order):
    xyz, tets = workloads.polar_tube(8, 4, 6, radius=0.01, length=0.03)
    rng = np.random.default_rng(80 + order)
    x0, x1 = degenerate_chords(xyz, tets, rng, 300, 0.002, dyadic=False)
    o, g, w = _run(xyz, tets, order, x0, x1, 1e-11)
    _compare(o, g, w)


def _compare(o, g, w):
    assert np.array_equal(g.get("TET"), w["tet"])
    assert np.array_equal(g.get("NCROSS"), w["ncross"])
    assert np.array_equal(g.get("HASH"), w["hash"])
    assert np.array_equal(g.get("X"), w["x"])
    assert np.array_equal(g.get("V"), w["v"])
    assert_elementwise(g.get("DG"), w["dg"], w["dg_abs"], 1e-12, "dg")
    assert_elementwise(g.get("RHO"), o.rho, o.rho_abs, 1e-12, "rho")
    d = g.diag()
    assert d["continuity_abs"] <= 1e-12 * d["continuity_ref"]
    assert w["ncross"].sum() > len(w["x"])
    g.close()

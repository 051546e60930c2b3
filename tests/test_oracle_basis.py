"""Pins of the oracle's mesh, quadrature and basis functions (no GPU).

Each check is fixed by something other than the oracle itself: closed-form
integrals, ranks and polynomial reproduction of the Appendix spaces,
finite-difference curls, inter-element continuity, the exact sequence, and
the linear-field reconstruction printed in Table tab:divblin.
"""

import itertools
import json
import math
import os

import numpy as np
import pytest

from oracle import assemble, basis, geometry, quadrature, topology
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


def _rand_tet(rng):
    while True:
        p = rng.normal(size=(4, 3))
        if abs(np.linalg.det(p[1:] - p[0])) > 0.3:
            return p


def _maps(p):
    g, c, vol = geometry.barycentric_maps(p, np.array([[0, 1, 2, 3]]))
    return g[0], c[0], vol[0]


def _rand_pts_in(p, n, rng):
    e = -np.log(rng.uniform(size=(n, 4)))
    lam = e / e.sum(axis=1, keepdims=True)
    return lam @ p


# ------------------------------------------------------------- quadrature
def test_tet_rule_monomials_closed_form():
    """int_ref l0^a l1^b l2^c l3^d = a! b! c! d! / (a+b+c+d+3)!"""
    lam, w = quadrature.tet_rule(4)
    assert abs(w.sum() - 1.0 / 6.0) < 1e-15
    for a, b, c, d in itertools.product(range(4), repeat=4):
        if a + b + c + d > 5:
            continue
        exact = (math.factorial(a) * math.factorial(b) * math.factorial(c)
                 * math.factorial(d) / math.factorial(a + b + c + d + 3))
        got = np.sum(w * lam[:, 0] ** a * lam[:, 1] ** b * lam[:, 2] ** c * lam[:, 3] ** d)
        assert abs(got - exact) <= 1e-15 + 1e-13 * exact


def test_gauss_legendre01_exact():
    for n in (1, 2, 4, 8):
        x, w = quadrature.gauss_legendre01(n)
        for k in range(2 * n):
            assert abs(np.sum(w * x ** k) - 1.0 / (k + 1)) < 1e-14


# --------------------------------------------------------------- topology
def test_c1_mesh_counts_and_euler():
    xyz, tets = workloads.kuhn_box(6, 6, 6, jitter=0.1, seed=1)
    t = topology.Topology(xyz, tets, 1)
    assert (t.n_tets, t.n_nodes, t.n_edges, t.n_faces) == (1296, 343, 1854, 2808)
    assert t.boundary_edge.sum() == 648 and t.boundary_face.sum() == 432
    assert t.n_nodes - t.n_edges + t.n_faces - t.n_tets == 1  # a ball
    vol = workloads.tet_volumes(xyz, tets)
    assert np.all(np.abs(vol) > 0.05 / 6 / 216)
    assert abs(np.abs(vol).sum() - 1.0) < 1e-12


def test_tube_mesh_counts():
    xyz, tets = workloads.polar_tube()
    t = topology.Topology(xyz, tets, 2)
    assert (t.n_tets, t.n_nodes, t.n_edges, t.n_faces) == (132480, 23409, 158360, 267432)
    assert t.n_nodes - t.n_edges + t.n_faces - t.n_tets == 1
    assert t.n1 == 851584 and t.n2 == 1199736
    assert np.all(np.abs(workloads.tet_volumes(xyz, tets)) > 0)


def test_dof_counts_match_appendix():
    gold = json.load(open(GOLDEN))["dof_counts_per_tet"]
    for k in (1, 2, 3):
        n0, n1, n2 = basis.n_local(k)
        assert (n0, n1, n2) == (gold[f"k{k}"]["w0"], gold[f"k{k}"]["w1"], gold[f"k{k}"]["w2"])
        if k < 3:
            assert len(basis.w1_spec(k)) == n1 and len(basis.w2_spec(k)) == n2
        else:
            from oracle import basis3
            assert len(basis3.w1_spec3()) == n1 and len(basis3.w2_spec3()) == n2
            assert len(basis3.w0_spec3()) == n0


def test_barycentric_maps():
    rng = np.random.default_rng(0)
    for _ in range(20):
        p = _rand_tet(rng)
        g, c, vol = _maps(p)
        lam = geometry.lam(g[None], c[None], p)
        assert np.allclose(lam, np.eye(4), atol=1e-14)
        assert abs(vol - abs(np.linalg.det(p[1:] - p[0])) / 6) < 1e-14 * vol
        x = rng.normal(size=(10, 3))
        assert np.allclose(geometry.lam(g[None], c[None], x).sum(axis=1), 1.0, atol=1e-14)


# ------------------------------------------------------------------ bases
def _values(fn, order, p, pts):
    g, c, _ = _maps(p)
    lam = geometry.lam(g[None], c[None], pts)
    gg = np.broadcast_to(g, (len(pts), 4, 3))
    return fn(order, lam, gg) if fn is not basis.w0 else fn(order, lam)


@pytest.mark.parametrize("order", [1, 2, 3])
def test_ranks(order):
    rng = np.random.default_rng(1)
    p = _rand_tet(rng)
    pts = _rand_pts_in(p, 60, rng)
    n0, n1, n2 = basis.n_local(order)
    w1 = _values(basis.w1, order, p, pts)
    w2 = _values(basis.w2, order, p, pts)
    assert np.linalg.matrix_rank(np.transpose(w1, (0, 2, 1)).reshape(-1, n1), tol=1e-9) == n1
    assert np.linalg.matrix_rank(np.transpose(w2, (0, 2, 1)).reshape(-1, n2), tol=1e-9) == n2
    w0 = _values(basis.w0, order, p, pts)
    assert np.linalg.matrix_rank(w0, tol=1e-9) == n0


def _in_span(vals, target):
    A = np.transpose(vals, (0, 2, 1)).reshape(-1, vals.shape[1])
    y = target.reshape(-1)
    x, *_ = np.linalg.lstsq(A, y, rcond=None)
    return np.max(np.abs(A @ x - y)) / max(1.0, np.max(np.abs(y)))


@pytest.mark.parametrize("order", [1, 2, 3])
def test_polynomial_reproduction(order):
    """W1 of order 1 spans the Whitney space {a + b x r}; order 2 spans all
    linear vector fields and gradients of quadratics (Nedelec first kind of
    degree 2).  W2 of order 1 spans {a + c r}; order 2 all linear fields."""
    rng = np.random.default_rng(2)
    p = _rand_tet(rng)
    pts = _rand_pts_in(p, 80, rng)
    w1 = _values(basis.w1, order, p, pts)
    w2 = _values(basis.w2, order, p, pts)
    for _ in range(5):
        a, bb = rng.normal(size=3), rng.normal(size=3)
        c0 = rng.normal()
        assert _in_span(w1, a + np.cross(bb, pts)) < 1e-12
        assert _in_span(w2, a + c0 * pts) < 1e-12
        if order == 3:
            # all quadratic vector fields (Nedelec / Raviart-Thomas of degree 3 contain P2^3)
            Q = rng.normal(size=(3, 3, 3))
            quad = np.einsum("kij,qi,qj->qk", Q, pts, pts) + pts @ rng.normal(size=(3, 3)) + a
            assert _in_span(w1, quad) < 1e-11
            assert _in_span(w2, quad) < 1e-11
        if order >= 2:
            G = rng.normal(size=(3, 3))
            lin = pts @ G.T + a
            assert _in_span(w1, lin) < 1e-12
            assert _in_span(w2, lin) < 1e-12
            S = rng.normal(size=(3, 3))
            S = S + S.T
            assert _in_span(w1, pts @ S + a) < 1e-12  # grad of a quadratic
        else:
            G = rng.normal(size=(3, 3))
            assert _in_span(w1, pts @ (G + G.T).T) > 1e-3  # not in the order-1 space
    w0 = _values(basis.w0, order, p, pts)
    assert np.allclose(w0.sum(axis=1), 1.0, atol=1e-13)  # partition of unity


@pytest.mark.parametrize("order", [1, 2, 3])
def test_curl_against_finite_differences(order):
    rng = np.random.default_rng(3)
    p = _rand_tet(rng)
    g, c, _ = _maps(p)
    pts = _rand_pts_in(p, 5, rng)
    h = 1e-5
    for x in pts:
        lamx = geometry.lam(g[None], c[None], x[None])
        cw = basis.curl_w1(order, lamx, g[None])[0]
        jac = np.zeros((cw.shape[0], 3, 3))  # d W_i[k] / d x_j
        for j in range(3):
            dx = np.zeros(3)
            dx[j] = h
            wp = basis.w1(order, geometry.lam(g[None], c[None], (x + dx)[None]), g[None])[0]
            wm = basis.w1(order, geometry.lam(g[None], c[None], (x - dx)[None]), g[None])[0]
            jac[:, :, j] = (wp - wm) / (2 * h)
        fd = np.stack([jac[:, 2, 1] - jac[:, 1, 2], jac[:, 0, 2] - jac[:, 2, 0],
                       jac[:, 1, 0] - jac[:, 0, 1]], axis=1)
        assert np.max(np.abs(fd - cw)) < 1e-6 * max(1.0, np.max(np.abs(cw)))
        dw = basis.div_w2(order, lamx, g[None])[0]
        dfd = np.zeros(dw.shape)
        for j in range(3):
            dx = np.zeros(3)
            dx[j] = h
            wp = basis.w2(order, geometry.lam(g[None], c[None], (x + dx)[None]), g[None])[0]
            wm = basis.w2(order, geometry.lam(g[None], c[None], (x - dx)[None]), g[None])[0]
            dfd += (wp[:, j] - wm[:, j]) / (2 * h)
        assert np.max(np.abs(dfd - dw)) < 1e-6 * max(1.0, np.max(np.abs(dw)))


@pytest.mark.parametrize("order", [1, 2, 3])
def test_exact_sequence_maps(order):
    d_loc, res_d = assemble.local_grad_map(order)
    c_loc, res_c = assemble.local_curl_map(order)
    tol = 1e-13 if order < 3 else 1e-12   # order-3 values reach (4 l)^3
    assert res_d < tol and res_c < tol
    assert np.max(np.abs(c_loc @ d_loc)) < tol  # curl grad = 0
    # affine invariance: the reference-tet coefficients hold on any tet
    rng = np.random.default_rng(4)
    for _ in range(5):
        p = _rand_tet(rng)
        pts = _rand_pts_in(p, 30, rng)
        w1 = _values(basis.w1, order, p, pts)
        w2 = _values(basis.w2, order, p, pts)
        g, c, _ = _maps(p)
        lam = geometry.lam(g[None], c[None], pts)
        gg = np.broadcast_to(g, (len(pts), 4, 3))
        gw0 = basis.grad_w0(order, lam, gg)
        cw1 = basis.curl_w1(order, lam, gg)
        assert np.max(np.abs(np.einsum("qik,ij->qjk", w1, d_loc) - gw0)) < 1e-12 * np.max(np.abs(gw0))
        assert np.max(np.abs(np.einsum("qfk,fj->qjk", w2, c_loc) - cw1)) < 1e-12 * np.max(np.abs(cw1))
    if order == 1:
        # lowest order: edge-node and face-edge incidence (Section III-A)
        for j, (s, t) in enumerate(topology.LOCAL_EDGES):
            col = np.zeros(4)
            col[s], col[t] = -1.0, 1.0
            assert np.allclose(d_loc[j], col)
        for f, (s, t, u) in enumerate(topology.LOCAL_FACES):
            row = np.zeros(6)
            row[topology.LOCAL_EDGES.index((s, t))] = 1
            row[topology.LOCAL_EDGES.index((t, u))] = 1
            row[topology.LOCAL_EDGES.index((s, u))] = -1
            assert np.allclose(c_loc[f], row)


@pytest.mark.parametrize("order", [1, 2, 3])
def test_interelement_continuity(order):
    """Tangential trace of sum e_i W1_i and normal trace of sum b_j W2_j agree
    from both sides of every interior face of a small jittered mesh."""
    xyz, tets = workloads.kuhn_box(2, 2, 2, jitter=0.15, seed=5)
    t = topology.Topology(xyz, tets, order)
    g, c, _ = geometry.barycentric_maps(t.xyz, t.tets)
    rng = np.random.default_rng(6)
    e = rng.normal(size=t.n1)
    b = rng.normal(size=t.n2)
    worst_t = worst_n = 0.0
    for f in np.nonzero(~t.boundary_face)[0]:
        verts = xyz[t.faces[f]]
        n = np.cross(verts[1] - verts[0], verts[2] - verts[0])
        n /= np.linalg.norm(n)
        pts = _rand_pts_in(np.vstack([verts, verts[0]]), 4, rng)
        owners = [tt for tt in range(t.n_tets) if f in t.tet_faces[tt]]
        vals = []
        for tt in owners:
            lam = geometry.lam(g[tt][None], c[tt][None], pts)
            gg = np.broadcast_to(g[tt], (len(pts), 4, 3))
            E = basis.combine(np.broadcast_to(e[t.dof1[tt]], (len(pts), t.dof1.shape[1])),
                              basis.w1(order, lam, gg))
            B = basis.combine(np.broadcast_to(b[t.dof2[tt]], (len(pts), t.dof2.shape[1])),
                              basis.w2(order, lam, gg))
            vals.append((E - np.outer(E @ n, n), B @ n))
        worst_t = max(worst_t, np.max(np.abs(vals[0][0] - vals[1][0])))
        worst_n = max(worst_n, np.max(np.abs(vals[0][1] - vals[1][1])))
    assert worst_t < 1e-10 and worst_n < 1e-10


@pytest.mark.parametrize("order", [1, 2, 3])
def test_global_maps_consistent_and_exact(order):
    xyz, tets = workloads.kuhn_box(3, 3, 3, jitter=0.1, seed=7)
    t = topology.Topology(xyz, tets, order)
    D = assemble.grad_matrix(t)   # raises if shared entities disagree
    C = assemble.curl_matrix(t)
    assert abs(C @ D).max() < 1e-13
    # D maps interior W0 DOFs onto free (non-PEC) W1 DOFs only
    Dint = D[:, np.nonzero(t.interior0)[0]]
    assert abs(Dint[np.nonzero(t.pec1)[0]]).max() == 0.0


def _project_w2(t, g, c, vol, field, order):
    """Galerkin (non-constrained) reconstruction [*mu^-1] b = f, Section III-C."""
    M2 = assemble.mass2(t, g, vol) * assemble.MU0
    lam_q, w_q = quadrature.tet_rule(4)
    f = np.zeros(t.n2)
    err_num = err_den = 0.0
    x_all = np.einsum("qk,tkd->tqd", lam_q, t.xyz[t.tets])
    for tt in range(t.n_tets):
        gg = np.broadcast_to(g[tt], (len(lam_q), 4, 3))
        w = basis.w2(order, lam_q, gg)
        F = field(x_all[tt])
        np.add.at(f, t.dof2[tt], 6 * vol[tt] * np.einsum("q,qik,qk->i", w_q, w, F))
    import scipy.sparse.linalg as spla
    bcoef = spla.spsolve(M2.tocsc(), f)
    div_max = 0.0
    for tt in range(t.n_tets):
        gg = np.broadcast_to(g[tt], (len(lam_q), 4, 3))
        w = basis.w2(order, lam_q, gg)
        Bh = np.einsum("i,qik->qk", bcoef[t.dof2[tt]], w)
        F = field(x_all[tt])
        err_num += 6 * vol[tt] * np.sum(w_q * np.sum((Bh - F) ** 2, axis=1))
        err_den += 6 * vol[tt] * np.sum(w_q * np.sum(F ** 2, axis=1))
        dv = basis.div_w2(order, lam_q, gg) @ bcoef[t.dof2[tt]]
        div_max = max(div_max, np.max(np.abs(dv)))
    return math.sqrt(err_num / err_den), div_max


def test_linear_field_reconstruction_table_divblin():
    """Table tab:divblin: B = y x^ + x y^ is reconstructed to machine precision
    at order 2 (printed 1.1049e-15) but not at order 1."""
    gold = json.load(open(GOLDEN))["linear_field_reconstruction"]
    xyz, tets = workloads.kuhn_box(4, 2, 2, lengths=gold["box_m"], jitter=0.1, seed=8)

    def field(x):
        return np.stack([x[:, 1], x[:, 0], np.zeros(len(x))], axis=1)

    for order, bound in ((2, 1e-13), (1, None)):
        t = topology.Topology(xyz, tets, order)
        g, c, vol = geometry.barycentric_maps(t.xyz, t.tets)
        err, div_max = _project_w2(t, g, c, vol, field, order)
        if bound:
            assert err < bound, err
            assert gold["error_B_nonconstrained"] < bound
            assert div_max < 1e-11
        else:
            assert err > 1e-4


def test_whitney_element_matrices_closed_form():
    """Order 1: int l_i l_j = V (1 + delta_ij) / 20 gives the Whitney mass
    matrix; curl w_ab = 2 grad l_a x grad l_b gives the curl-curl matrix."""
    rng = np.random.default_rng(11)
    for _ in range(5):
        p = _rand_tet(rng)
        t = topology.Topology(p, np.array([[0, 1, 2, 3]]), 1)
        g, c, vol = geometry.barycentric_maps(t.xyz, t.tets)
        M = assemble.mass1(t, g, vol).toarray() / assemble.EPS0
        K = assemble.curlcurl(t, g, vol).toarray() * assemble.MU0
        G = g[0] @ g[0].T
        V = vol[0]

        def ll(i, j):
            return V * (1.0 + (i == j)) / 20.0

        for I, (a, b) in enumerate(topology.LOCAL_EDGES):
            for J, (cc, d) in enumerate(topology.LOCAL_EDGES):
                m = (G[b, d] * ll(a, cc) - G[b, cc] * ll(a, d)
                     - G[a, d] * ll(b, cc) + G[a, cc] * ll(b, d))
                k = 4.0 * V * (G[a, cc] * G[b, d] - G[a, d] * G[b, cc])
                assert abs(M[I, J] - m) < 1e-13 * np.abs(M).max()
                assert abs(K[I, J] - k) < 1e-13 * np.abs(K).max()


@pytest.mark.parametrize("order", [1, 2, 3])
def test_global_mass_and_curlcurl_energies(order):
    """For E = grad(phi) with phi linear, e = D phi_h gives e^T M e =
    eps0 |grad phi|^2 Vol and K e = 0; the L2 projection of E = (-y, x, 0)/2
    (curl E = z^) gives e^T K e = Vol / mu0 and e^T M e = eps0 int |E|^2."""
    xyz, tets = workloads.kuhn_box(3, 3, 3, jitter=0.1, seed=12)
    t = topology.Topology(xyz, tets, order)
    g, c, vol = geometry.barycentric_maps(t.xyz, t.tets)
    M = assemble.mass1(t, g, vol)
    K = assemble.curlcurl(t, g, vol)
    D = assemble.grad_matrix(t)
    k = np.array([0.3, -1.2, 0.7])
    if order == 1:
        phi = xyz @ k
    elif order == 2:
        mid = 0.5 * (xyz[t.edges[:, 0]] + xyz[t.edges[:, 1]])
        phi = np.concatenate([xyz @ k, mid @ k])
    else:
        # W0 lattice points: nodes, (2a+b)/3 and (a+2b)/3 per edge, face centroids
        a, b = xyz[t.edges[:, 0]], xyz[t.edges[:, 1]]
        ep = np.stack([(2 * a + b) / 3, (a + 2 * b) / 3], axis=1).reshape(-1, 3)
        fc = xyz[t.faces].mean(axis=1)
        phi = np.concatenate([xyz @ k, ep @ k, fc @ k])
    e = D @ phi
    assert abs(e @ (M @ e) - assemble.EPS0 * (k @ k) * 1.0) < 1e-12 * assemble.EPS0 * (k @ k)
    assert np.abs(K @ e).max() < 1e-10 * np.abs(K).max() * np.abs(e).max()
    lam_q, w_q = quadrature.tet_rule(4)
    f = np.zeros(t.n1)
    x_all = np.einsum("qk,tkd->tqd", lam_q, t.xyz[t.tets])
    for tt in range(t.n_tets):
        w = basis.w1(order, lam_q, np.broadcast_to(g[tt], (len(lam_q), 4, 3)))
        F = np.stack([-x_all[tt][:, 1], x_all[tt][:, 0], 0 * x_all[tt][:, 0]], axis=1) * 0.5
        np.add.at(f, t.dof1[tt], 6 * vol[tt] * np.einsum("q,qik,qk->i", w_q, w, F))
    import scipy.sparse.linalg as spla
    e = spla.spsolve((M / assemble.EPS0).tocsc(), f)
    assert abs(e @ (K @ e) * assemble.MU0 - 1.0) < 1e-12
    exact = (1.0 / 3.0 + 1.0 / 3.0) / 4.0  # int over the unit cube of (x^2 + y^2) / 4
    assert abs(e @ (M @ e) / assemble.EPS0 - exact) < 1e-12

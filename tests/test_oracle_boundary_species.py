"""Pins of the oracle's impedance boundary and multi-species stepping.

Impedance (Section II eq. impedanceBC, Section III-A [*_I]): the surface
matrix is checked against closed forms that do not use the basis -- the
energy Y int |n x E|^2 dS of fields the order-p W1 space reproduces exactly --
and the trapezoid step against its discrete energy balance.  Species (the
paper's ion-electron plasma ball): splitting one species into two identical
ones changes nothing, and charge stays conserved with ions and electrons.
"""

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads
from oracle import assemble, geometry, quadrature, sim as osim, topology

Q_E = 1.602176634e-19
M_E = 9.1093837015e-31
M_SR = 87.62 * 1.66053906660e-27


def tags_on_plane(xyz, tets, axis, value, tol=1e-12):
    """Tag 1 (impedance) on tet faces lying in the plane x[axis] = value."""
    tets = np.asarray(tets)
    tag = np.zeros(tets.shape, dtype=np.int32)
    for i in range(4):
        others = np.delete(tets, i, axis=1)
        on = np.all(np.abs(xyz[others][:, :, axis] - value) < tol, axis=1)
        tag[on, i] = 1
    return tag


def _box(order, n=3, seed=7):
    xyz, tets = workloads.kuhn_box(n, n, n, jitter=0.1, seed=seed)
    tag = tags_on_plane(xyz, tets, 0, 1.0)
    t = topology.Topology(xyz, tets, order, tag)
    g, c, vol = geometry.barycentric_maps(t.xyz, t.tets)
    return xyz, tets, tag, t, g, vol


@pytest.mark.parametrize("order", [1, 2])
def test_impedance_faces_and_free_dofs(order):
    xyz, tets, tag, t, g, vol = _box(order)
    assert t.imp_face.sum() == 2 * 3 * 3          # the x = 1 square, 2 triangles per cell
    assert np.all(t.boundary_face[t.imp_face])
    I = assemble.impedance(t, g)
    assert abs(I - I.T).max() <= 1e-14 * abs(I).max()
    w = np.linalg.eigvalsh(I.toarray())
    assert w.min() >= -1e-12 * w.max()
    # I couples only W1 DOFs that live on impedance faces
    on_imp = np.zeros(t.n1, dtype=bool)
    for f in np.nonzero(t.imp_face)[0]:
        tt, i = [int(a[0]) for a in np.nonzero(t.tet_faces == f)]
        loc = [j for j, (a, b) in enumerate(topology.LOCAL_EDGES) if a != i and b != i]
        if order == 1:
            on_imp[t.dof1[tt, loc]] = True
        else:
            on_imp[t.dof1[tt, [2 * j for j in loc] + [2 * j + 1 for j in loc]]] = True
            on_imp[t.dof1[tt, [12 + 2 * i, 13 + 2 * i]]] = True
    rows = np.unique(I.nonzero()[0])
    assert np.all(on_imp[rows])
    # interior edges of the impedance square are free; its rim (shared with PEC faces) is not
    assert np.any(on_imp & t.free1)
    if order == 2:
        fid = np.nonzero(t.imp_face)[0]
        assert np.all(t.free1[2 * t.n_edges + 2 * fid])


@pytest.mark.parametrize("order", [1, 2, 3])
def test_impedance_energy_of_uniform_field(order):
    """E = k (e = D phi, phi = k.x, exact at every order): e^T I e equals
    Y0 |n x k|^2 times the area of the impedance face (the unit square x=1)."""
    xyz, tets, tag, t, g, vol = _box(order)
    I = assemble.impedance(t, g)
    D = assemble.grad_matrix(t)
    k = np.array([0.3, -1.2, 0.7])
    if order == 1:
        phi = t.xyz @ k
    elif order == 2:
        mid = 0.5 * (t.xyz[t.edges[:, 0]] + t.xyz[t.edges[:, 1]])
        phi = np.concatenate([t.xyz @ k, mid @ k])
    else:  # the cubic lattice: nodes, two points per edge (nearer the lower vertex first), face centroids
        a, b = t.xyz[t.edges[:, 0]], t.xyz[t.edges[:, 1]]
        ep = np.stack([(2 * a + b) / 3, (a + 2 * b) / 3], axis=1).reshape(-1, 3)
        fc = t.xyz[t.faces].mean(axis=1)
        phi = np.concatenate([t.xyz @ k, ep @ k, fc @ k])
    e = D @ phi
    want = assemble.Y0 * (k[1] ** 2 + k[2] ** 2) * 1.0
    assert abs(e @ (I @ e) - want) <= 1e-12 * want


@pytest.mark.parametrize("order", [1, 2, 3])
def test_impedance_energy_of_rotational_field(order):
    """E = (-y, x, 0) / 2 (in the W1 span at every order; its L2 projection is
    exact): on x = 1, |n x E|^2 = E_y^2 + E_z^2 = 1/4, so e^T I e = Y0 / 4."""
    xyz, tets, tag, t, g, vol = _box(order)
    I = assemble.impedance(t, g)
    M = assemble.mass1(t, g, vol) / assemble.EPS0
    lam_q, w_q = quadrature.tet_rule(4)
    f = np.zeros(t.n1)
    from oracle import basis
    x_all = np.einsum("qk,tkd->tqd", lam_q, t.xyz[t.tets])
    for tt in range(t.n_tets):
        w = basis.w1(order, lam_q, np.broadcast_to(g[tt], (len(lam_q), 4, 3)))
        F = np.stack([-x_all[tt][:, 1], x_all[tt][:, 0], 0 * x_all[tt][:, 0]], axis=1) * 0.5
        np.add.at(f, t.dof1[tt], 6 * vol[tt] * np.einsum("q,qik,qk->i", w_q, w, F))
    e = spla.spsolve(M.tocsc(), f)
    assert abs(e @ (I @ e) - assemble.Y0 / 4.0) <= 1e-11 * assemble.Y0


def test_tri_rule_exactness():
    """int_T x^a y^b over the reference triangle = a! b! / (a + b + 2)!."""
    from math import factorial
    lam, w = quadrature.tri_rule(4)
    assert abs(w.sum() - 0.5) < 1e-15
    for a in range(5):
        for b in range(5 - a):
            got = np.sum(w * lam[:, 1] ** a * lam[:, 2] ** b)
            want = factorial(a) * factorial(b) / factorial(a + b + 2)
            assert abs(got - want) < 1e-15


def _quiet_sim(order, tag, dt, seed):
    xyz, tets = workloads.kuhn_box(3, 3, 3, jitter=0.1, seed=7)
    s = osim.Sim(xyz, tets, order, -Q_E, M_E, 0.0, bface_tag=tag)
    rng = np.random.default_rng(seed)
    x, tet = workloads.sample_uniform_in_tets(xyz, tets, 10, rng)
    s.set_particles(x, workloads.maxwellian(10, 1e5, rng), tet)   # weight 0: no sources
    t = s.topo
    s.e = workloads.random_dof_vector(t.n1, 1.0, rng, t.pec1)
    s.e_prev = s.e.copy()
    s.b = workloads.random_dof_vector(t.n2, 1e-8, rng)
    return s


@pytest.mark.parametrize("order", [1, 2])
def test_trapezoid_energy_balance_with_impedance(order):
    """Without sources the trapezoid step loses exactly dt ebar.I ebar of the
    energy e.[*eps]e/2 + b.[*mu^-1]b/2 through the impedance face, and keeps
    it (to rounding) with PEC walls only."""
    xyz, tets = workloads.kuhn_box(3, 3, 3, jitter=0.1, seed=7)
    tag = tags_on_plane(xyz, tets, 0, 1.0)
    dt = 2e-10
    s = _quiet_sim(order, tag, dt, 3)
    for _ in range(3):
        w0, e0 = s.energy(), s.e.copy()
        s.step(dt)
        eb = 0.5 * (s.e + e0)
        loss = dt * eb @ (s.I @ eb)
        assert loss > 0.0
        assert abs((w0 - s.energy()) - loss) <= 1e-9 * w0
    p = _quiet_sim(order, None, dt, 3)
    w_start = p.energy()
    for _ in range(3):
        p.step(dt)
    assert abs(p.energy() - w_start) <= 1e-10 * w_start


@pytest.mark.parametrize("order", [1, 2])
def test_species_split_is_the_same_species(order):
    """Two species with the same q, m and weight are one species in two parts."""
    cfg = workloads.make_config(0, n_particles=600)
    rng = np.random.default_rng(5)
    one = osim.Sim(cfg["xyz"], cfg["tets"], order, cfg["q"], cfg["m"], cfg["weight"], cfg["B0"])
    one.set_particles(cfg["x"], cfg["v"], cfg["tet"])
    two = osim.Sim(cfg["xyz"], cfg["tets"], order, cfg["q"], cfg["m"], cfg["weight"], cfg["B0"])
    h = 250
    two.set_species([dict(q=cfg["q"], m=cfg["m"], weight=cfg["weight"], x=cfg["x"][:h], v=cfg["v"][:h],
                          tet=cfg["tet"][:h]),
                     dict(q=cfg["q"], m=cfg["m"], weight=cfg["weight"], x=cfg["x"][h:], v=cfg["v"][h:],
                          tet=cfg["tet"][h:])])
    e = workloads.random_dof_vector(one.topo.n1, 1e3, rng, one.topo.pec1)
    for s in (one, two):
        s.e, s.e_prev = e.copy(), e.copy()
    a, b = one.step(cfg["dt"]), two.step(cfg["dt"])
    assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["tet"], b["tet"])
    assert np.abs(a["dg"] - b["dg"]).max() <= 1e-13 * np.abs(a["dg"]).max()
    assert np.abs(one.rho - two.rho).max() <= 1e-13 * np.abs(one.rho).max()


@pytest.mark.parametrize("order", [1, 2])
def test_ions_and_electrons_conserve_charge(order):
    """Sr+ ions and electrons (the plasma-ball species): the ion moves with
    its own q/m, the currents add, and Delta rho = D^T Delta g holds for the
    total charge; the ion charge enters rho with its sign."""
    xyz, tets = workloads.kuhn_box(4, 4, 4, jitter=0.1, seed=9)
    rng = np.random.default_rng(6)
    n = 300
    xe, te = workloads.sample_uniform_in_tets(xyz, tets, n, rng)
    xi, ti = workloads.sample_uniform_in_tets(xyz, tets, n, rng)
    ve = workloads.maxwellian(n, 2e6, rng)
    vi = workloads.maxwellian(n, 2e4, rng)
    s = osim.Sim(xyz, tets, order, -Q_E, M_E, 1e5)
    s.set_species([dict(q=-Q_E, m=M_E, weight=1e5, x=xe, v=ve, tet=te),
                   dict(q=Q_E, m=M_SR, weight=1e5, x=xi, v=vi, tet=ti)])
    t = s.topo
    s.e = workloads.random_dof_vector(t.n1, 1e3, rng, t.pec1)
    s.e_prev = s.e.copy()
    only_e = osim.Sim(xyz, tets, order, -Q_E, M_E, 1e5)
    only_e.set_particles(xe, ve, te)
    assert np.all(s.rho[:t.n_nodes] * 0 == 0)
    w = s.step(1e-9)
    c = w["continuity"][t.interior0]
    assert np.linalg.norm(c) <= 1e-13 * np.linalg.norm(w["drho"][t.interior0])
    # the ions' own share: same rho as an ion-only measurement
    ion_rho = s.rho - osim.particles.measure_rho(t, s.g, s.c, w["x"][:n], w["tet"][:n], -Q_E * 1e5)
    direct = osim.particles.measure_rho(t, s.g, s.c, w["x"][n:], w["tet"][n:], Q_E * 1e5)
    assert np.abs(ion_rho - direct).max() <= 1e-12 * np.abs(direct).max()
    assert direct.sum() > 0

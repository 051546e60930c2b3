"""Pins of the oracle's Adams-Bashforth push on the quartic path (Section
III-B, last paragraph).

* the AB coefficients are the textbook ones and the path ends at the AB
  update (x(1) = x^n + dt sum beta_j v^{n-j}, x'(0) = dt v^n);
* with no field and a constant velocity the path is the straight chord, so
  the walk and the current equal the straight-chord oracle's;
* in a uniform B the gyration error falls as dt^4 (closed-form orbit);
* on curved paths through many tets, Delta rho = D^T Delta g holds and the
  current equals a brute-force fine-step path integral;
* at a wall the rest of the path is mirrored: the end point is the mirror
  image of the unreflected end point.
"""

import numpy as np
import pytest

import workloads
from oracle import ab4, assemble, basis, geometry, particles, sim as osim, topology

Q_E = 1.602176634e-19
M_E = 9.1093837015e-31


def test_ab_tables_and_path_ends():
    b4, g4 = ab4.ab_tables(4)
    assert np.allclose(b4 * 24.0, [55.0, -59.0, 37.0, -9.0], rtol=0, atol=1e-13)
    for k in (1, 2, 3, 4):
        b, g = ab4.ab_tables(k)
        assert np.allclose(g.sum(axis=1), b, rtol=0, atol=1e-15)   # gam_j(1) = beta_j
        assert np.all(g[:, 0] == 0.0)                              # path starts at x^n
        assert g[0, 1] == 1.0 and np.all(g[1:, 1] == 0.0)          # x'(0) = dt v^n
    rng = np.random.default_rng(1)
    x = rng.standard_normal((5, 3))
    vh = rng.standard_normal((4, 5, 3))
    C = ab4.path_coeffs(x, vh, 0.1, 4)
    end = ab4._horner(C, np.ones(5))
    want = x + 0.1 * ((b4[0] * vh[0] + b4[1] * vh[1]) + (b4[2] * vh[2] + b4[3] * vh[3]))
    assert np.abs(end - want).max() < 1e-14


@pytest.mark.parametrize("order", [1, 2])
def test_constant_velocity_is_the_straight_chord(order):
    xyz, tets = workloads.kuhn_box(4, 4, 4, jitter=0.1, seed=3)
    t = topology.Topology(xyz, tets, order)
    g, c, _ = geometry.barycentric_maps(t.xyz, t.tets)
    rng = np.random.default_rng(2)
    n = 200
    x, tet = workloads.sample_uniform_in_tets(xyz, tets, n, rng)
    v = rng.standard_normal((n, 3)) * 0.06
    dt = 1.0
    vh = np.broadcast_to(v, (3, n, 3)).copy()
    ah = np.zeros((3, n, 3))
    zero = np.zeros((n, 3))
    r = ab4.step(t, g, c, x, v, tet, vh, ah, 3, zero, zero, -1.0, 1.0, 2.0, dt, t.n1)
    x1 = x + dt * v
    xe, ve, te, dg, nc, hs, st, _ = particles.walk_deposit(t, g, c, x, x1, v, tet, 2.0, t.n1)
    moved = nc > 0
    assert moved.mean() > 0.3
    assert np.abs(r["x"] - xe).max() < 1e-12
    assert np.array_equal(r["tet"], te)
    assert np.array_equal(r["ncross"], nc)
    assert np.abs(r["dg"] - dg).max() <= 1e-12 * np.abs(dg).max()


def _gyration_error(dt, n_steps):
    """One electron in B = B0 z (no self field), AB4 from exact history;
    returns |x - x_exact| after n_steps."""
    xyz, tets = workloads.kuhn_box(2, 2, 2, lengths=(4.0, 4.0, 4.0))
    s = osim.Sim(xyz, tets, 1, -Q_E, M_E, 0.0, B0=(0.0, 0.0, 1e-3), push="ab4")
    wc = Q_E * 1e-3 / M_E                      # cyclotron frequency
    R = 0.5
    center = np.array([2.0, 2.0, 2.0])
    def state(time):
        ph = wc * time                         # electrons gyrate counter-clockwise about +z
        pos = center + R * np.array([np.cos(ph), np.sin(ph), 0.0])
        vel = R * wc * np.array([-np.sin(ph), np.cos(ph), 0.0])
        acc = -R * wc * wc * np.array([np.cos(ph), np.sin(ph), 0.0])
        return pos, vel, acc
    x0, v0, _ = state(0.0)
    tet = np.array([int(np.argmax(np.all(geometry.lam(s.g, s.c, np.broadcast_to(x0, (len(s.g), 3))) >= 0, axis=1)))])
    s.set_particles(x0[None], v0[None], tet)
    for j in range(3):
        _, vj, aj = state(-(j + 1) * dt)
        s.vh[j, 0], s.ah[j, 0] = vj, aj
    s.hcount = 3
    for _ in range(n_steps):
        s.step(dt)
    xe, _, _ = state(n_steps * dt)
    return np.linalg.norm(s.x[0] - xe)


def test_ab4_gyration_converges_at_fourth_order():
    wc = Q_E * 1e-3 / M_E
    period = 2 * np.pi / wc
    e1 = _gyration_error(period / 64, 64)
    e2 = _gyration_error(period / 128, 128)
    assert 12.0 < e1 / e2 < 20.0
    assert e2 < 1e-5


def _curved_setup(order, seed, n=150):
    xyz, tets = workloads.kuhn_box(4, 4, 4, jitter=0.1, seed=seed)
    s = osim.Sim(xyz, tets, order, -Q_E, M_E, 1e4, B0=(0.0, 0.0, 2e-4), push="ab4")
    rng = np.random.default_rng(seed)
    x, tet = workloads.sample_uniform_in_tets(xyz, tets, n, rng)
    s.set_particles(x, workloads.maxwellian(n, 2e7, rng), tet)
    t = s.topo
    s.e = workloads.random_dof_vector(t.n1, 1e2, rng, t.pec1)
    s.e_prev = s.e.copy()
    return s


@pytest.mark.parametrize("order", [1, 2])
def test_curved_paths_conserve_charge(order):
    s = _curved_setup(order, 11)
    t = s.topo
    crossings = 0
    for k in range(5):
        w = s.step(2e-9)
        assert w["order"] == min(4, k + 1)
        crossings += w["ncross"].sum()
        c = w["continuity"][t.interior0]
        assert np.linalg.norm(c) <= 1e-13 * np.linalg.norm(w["drho"][t.interior0])
    assert crossings > 500


def _brute_force_current(t, g, c, C, qw, n_fine=6000):
    """q w int W1 . x'(s) ds by the midpoint rule on n_fine steps, the owning
    tet of every step's midpoint found by trying every tet."""
    dg = np.zeros(t.n1)
    s = (np.arange(n_fine) + 0.5) / n_fine
    for p in range(len(C)):
        pts = ab4._horner(np.broadcast_to(C[p], (n_fine,) + C[p].shape), s)
        dx = ab4._horner_deriv(np.broadcast_to(C[p], (n_fine,) + C[p].shape), s) / n_fine
        lam = np.einsum("tik,qk->qti", g, pts) + c[None]
        owner = np.argmax(lam.min(axis=2), axis=1)
        L = lam[np.arange(n_fine), owner]
        gg = g[owner]
        W = basis.w1(t.order, L, gg)
        np.add.at(dg, t.dof1[owner].ravel(), (qw * np.einsum("qjk,qk->qj", W, dx)).ravel())
    return dg


@pytest.mark.parametrize("order", [1, 2])
def test_curved_current_matches_brute_force(order):
    s = _curved_setup(order, 12, n=8)
    t = s.topo
    for _ in range(3):                           # fill the history: AB4 on the last step
        s.step(2e-9)
    vhist = np.concatenate([s.v[None], s.vh[:3]], axis=0)
    C = ab4.path_coeffs(s.x, vhist, 2e-9, 4)
    free_end = ab4._horner(C, np.ones(len(C)))
    g0 = geometry.lam(s.g[None], s.c[None], free_end[:, None, :])   # all tets: does the end stay inside?
    keep = np.nonzero(np.any(np.all(g0 >= 0.0, axis=2), axis=1))[0]  # paths that meet no wall
    E, B = particles.gather(t, s.g, s.c, s.e, s.b, s.B0, s.x[keep], s.tet[keep])
    r = ab4.step(t, s.g, s.c, s.x[keep], s.v[keep], s.tet[keep], s.vh[:, keep], s.ah[:, keep], s.hcount,
                 E, B, -Q_E, M_E, -Q_E * 1e4, 2e-9, t.n1)
    assert r["order"] == 4 and r["ncross"].sum() >= 3
    assert np.abs(r["x"] - free_end[keep]).max() < 1e-12
    ref = _brute_force_current(t, s.g, s.c, C[keep], -Q_E * 1e4)
    assert np.linalg.norm(r["dg"] - ref) <= 5e-3 * np.linalg.norm(ref)


def test_wall_mirror_of_the_path():
    xyz, tets = workloads.kuhn_box(3, 3, 3)
    t = topology.Topology(xyz, tets, 1)
    g, c, _ = geometry.barycentric_maps(t.xyz, t.tets)
    x = np.array([[0.9, 0.5, 0.5]])
    tet = np.array([int(np.argmax(np.all(geometry.lam(g, c, np.broadcast_to(x[0], (len(g), 3))) >= 0, axis=1)))])
    v = np.array([[0.3, 0.05, 0.0]])
    a = np.array([[0.0, 0.2, 0.0]])
    vh = np.stack([v - a * j for j in (1, 2, 3)])
    ah = np.broadcast_to(a, (3, 1, 3)).copy()
    zero = np.zeros((1, 3))
    r = ab4.step(t, g, c, x, v, tet, vh, ah, 3, zero, zero, 0.0, 1.0, 1.0, 1.0, t.n1)
    vhist = np.concatenate([v[None], vh], axis=0)
    free_end = ab4._horner(ab4.path_coeffs(x, vhist, 1.0, 4), np.ones(1))[0]
    assert free_end[0] > 1.0                      # the unreflected path leaves through x = 1
    want = free_end.copy()
    want[0] = 2.0 - free_end[0]
    assert np.abs(r["x"][0] - want).max() < 1e-12
    assert r["v"][0, 0] < 0.0 and r["vh"][0, 0, 0] < 0.0   # velocity and history mirrored
    assert r["ncross"][0] >= 1

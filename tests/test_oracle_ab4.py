"""Pins of the oracle's Adams-Bashforth push on the quartic path (Section
III-B, last paragraph).

* the AB coefficients are the textbook ones and the path ends at the AB
  update (x(1) = x^n + dt sum beta_j v^{n-j}, x'(0) = dt v^n);
* with no field and a constant velocity the path is the straight chord, so
  the walk and the current equal the straight-chord oracle's;
* in a uniform B the gyration error falls as dt^4 (closed-form orbit);
* the crossing of a face is the first sign change of lambda_i(x(s)) to
  negative: closed-form roots, a tangent path that touches a face before it
  crosses, a path that dips through a face and back inside one eighth of the
  step, and bisection on densely sampled random quartics;
* on curved paths through many tets, Delta rho = D^T Delta g holds and the
  current equals a brute-force path integral split at crossings found by
  bisection on brute-force point location;
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


def _owner(g, c, x):
    """Tet containing x, by trying every tet (largest smallest barycentric)."""
    lam = np.einsum("tik,k->ti", g, x) + c
    return int(np.argmax(lam.min(axis=1)))


def _brute_force_current(t, g, c, C, qw, n_fine=2000, n_gl=8):
    """q w int W1 . x'(s) ds along each path, split where the owning tet
    changes: owners of n_fine + 1 sample points by brute-force point location,
    each change located by 60 bisections on the owner, each piece integrated
    by the n_gl-point Gauss-Legendre rule (exact: degree <= 4p + 3 < 2 n_gl)."""
    xq, wq = np.polynomial.legendre.leggauss(n_gl)
    xq, wq = 0.5 * (xq + 1.0), 0.5 * wq
    dg = np.zeros(t.n1)
    grid = np.linspace(0.0, 1.0, n_fine + 1)
    for p in range(len(C)):
        Cp = C[p][None]
        at = lambda s: ab4._horner(Cp, np.array([s]))[0]
        own = [_owner(g, c, at(s)) for s in grid]
        cuts = [0.0]
        pieces = [own[0]]
        for k in range(n_fine):
            if own[k + 1] == own[k]:
                continue
            lo, hi = grid[k], grid[k + 1]
            for _ in range(60):
                mid = 0.5 * (lo + hi)
                if _owner(g, c, at(mid)) == own[k]:
                    lo = mid
                else:
                    hi = mid
            cuts.append(0.5 * (lo + hi))
            pieces.append(own[k + 1])
        cuts.append(1.0)
        for j, T in enumerate(pieces):
            a, b = cuts[j], cuts[j + 1]
            s = a + (b - a) * xq
            pts = ab4._horner(np.broadcast_to(Cp, (len(s),) + C[p].shape), s)
            dx = ab4._horner_deriv(np.broadcast_to(Cp, (len(s),) + C[p].shape), s)
            lam = np.einsum("ik,qk->qi", g[T], pts) + c[T][None]
            W = basis.w1(t.order, lam, np.broadcast_to(g[T], (len(s),) + g[T].shape))
            contrib = qw * (b - a) * np.einsum("q,qjk,qk->j", wq, W, dx)
            np.add.at(dg, t.dof1[T], contrib)
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
    assert np.linalg.norm(r["dg"] - ref) <= 1e-12 * np.linalg.norm(ref)


def _poly_from_roots(roots, lead=1.0):
    return lead * np.polynomial.polynomial.polyfromroots(roots)


def test_first_exit_closed_forms():
    fe = ab4.first_exit
    assert fe([0.3, -1.0], 0.0, False) == 0.3                        # linear: lambda = 0.3 - s
    # touches the face at s = 1/4 (double root, stays inside), crosses at 3/4:
    # 4 (s - 1/4)^2 (3/4 - s), dyadic coefficients
    assert abs(fe([0.1875, -1.75, 5.0, -4.0], 0.0, False) - 0.75) < 1e-12
    # out and back inside one eighth of the step: (s - 0.3)(s - 0.34); every
    # eighth of the step is inside, the crossing is still found
    c = _poly_from_roots([0.3, 0.34])
    assert all(np.polyval(c[::-1], j / 8.0) > 0.0 for j in range(9))
    assert abs(fe(c, 0.0, False) - 0.3) < 1e-12
    assert fe(c, 0.32, False) == 0.32                               # starts outside: leaves at s0
    # closed-form root of s^2 - s + 0.21 (0.21 is not a binary fraction)
    want = (1.0 - np.sqrt(1.0 - 4.0 * 0.21)) / 2.0
    assert abs(fe([0.21, -1.0, 1.0], 0.0, False) - want) < 1e-15
    # four roots: the first negative piece after s0
    c = _poly_from_roots([0.1, 0.2, 0.6, 0.9])
    assert abs(fe(c, 0.0, False) - 0.1) < 1e-12
    assert fe(c, 0.15, False) == 0.15                                # negative at s0
    assert abs(fe(c, 0.4, False) - 0.6) < 1e-12
    # entry face (vanishes at s0): enters at 0.2, leaves at 0.7
    c = _poly_from_roots([0.2, 0.7], -1.0)
    assert abs(fe(c, 0.2, True) - 0.7) < 1e-12
    c_noisy = c.copy()
    c_noisy[0] += 1e-17                                              # lambda(s0) off by rounding
    assert abs(fe(c_noisy, 0.2, True) - 0.7) < 1e-12
    assert fe(-c, 0.2, True) == 0.2                                  # turns back at once
    assert fe([1.0, 0.0, 1.0], 0.0, False) == np.inf                 # stays positive
    assert fe([1.0, -1.0], 0.0, False) == np.inf                     # ends on the face: stays
    assert fe([0.25, -1.0, 1.0], 0.0, False) == np.inf               # touches at 1/2 only


def test_first_exit_matches_bisection_on_random_quartics():
    """First sign change found by dense sampling and bisection (no root
    finder), on quartics whose roots are at least 1e-3 apart."""
    rng = np.random.default_rng(4)
    grid = np.linspace(0.0, 1.0, 20001)
    checked = 0
    for _ in range(300):
        k = int(rng.integers(1, 5))
        roots = np.sort(rng.uniform(-0.3, 1.3, size=k))
        if k > 1 and np.diff(roots).min() < 1e-3:
            continue
        c = _poly_from_roots(roots, rng.choice([-1.0, 1.0]) * 10.0 ** rng.uniform(-2, 2))
        s0 = float(rng.choice([0.0, rng.uniform(0.0, 0.8)]))
        pts = grid[grid >= s0]
        f = np.polynomial.polynomial.polyval(pts, c)
        neg = np.nonzero(f < 0.0)[0]
        if neg.size == 0:
            want = np.inf
        elif neg[0] == 0:
            want = s0
        else:
            lo, hi = pts[neg[0] - 1], pts[neg[0]]
            for _ in range(80):
                mid = 0.5 * (lo + hi)
                if np.polynomial.polynomial.polyval(mid, c) < 0.0:
                    hi = mid
                else:
                    lo = mid
            want = 0.5 * (lo + hi)
        got = ab4.first_exit(c, s0, False)
        if np.isinf(want):
            assert got == np.inf
        else:
            assert abs(got - want) < 1e-12
            checked += 1
    assert checked > 100


def test_dip_within_one_eighth_is_two_crossings():
    """A path that leaves its tet through a face and comes back inside one
    eighth of the step crosses twice, at the roots of its height above the
    face (closed form), and ends in the tet it started in."""
    xyz, tets = workloads.kuhn_box(2, 2, 2)
    t = topology.Topology(xyz, tets, 1)
    g, c, _ = geometry.barycentric_maps(t.xyz, t.tets)
    # z(s) = 0.5 + 0.15 (s - 0.3)(s - 0.34): below the plane z = 0.5 on (0.3, 0.34)
    C0 = np.array([0.2, 0.1, 0.5 + 0.15 * 0.102])
    C1 = np.array([0.0, 0.0, -0.15 * 0.64])
    C2 = np.array([0.0, 0.0, 0.15])
    x = C0[None]
    v0 = C1[None]                                  # AB2 with dt = 1: C1 = v^n, C2 = (v^n - v^{n-1}) / 2
    vh = np.zeros((3, 1, 3))
    vh[0] = v0 - 2.0 * C2[None]
    tet = np.array([_owner(g, c, C0)])
    zero = np.zeros((1, 3))
    trace = []
    r = ab4.step(t, g, c, x, v0, tet, vh, np.zeros((3, 1, 3)), 1, zero, zero, 0.0, 1.0, 1.0, 1.0, t.n1,
                 trace=trace)
    assert r["order"] == 2
    assert r["ncross"][0] == 2 and r["tet"][0] == tet[0]
    (p0, t0, f0, s_out), (p1, t1, f1, s_back) = trace
    assert t0 == tet[0] and t1 == t.tet2tet[tet[0], f0]
    assert abs(s_out - 0.3) < 1e-12 and abs(s_back - 0.34) < 1e-12
    assert np.abs(r["x"][0] - (C0 + C1 + C2)).max() < 1e-15
    ref = _brute_force_current(t, g, c, np.stack([C0, C1, C2])[None], 1.0)
    assert np.linalg.norm(r["dg"] - ref) <= 1e-12 * np.linalg.norm(ref)


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

"""Pins of the oracle's absorbing and injecting walls (the paper is silent on
particle walls; its drift-tube beam enters at one end) and of the
counter-based generator they draw from."""

import numpy as np
import pytest

import workloads
from oracle import geometry, inject, particles, sim as osim, topology


def test_splitmix64_published_value():
    """SplitMix64 seeded with 0: its first output is 0xE220A8397B1DCDAF
    (Steele, Lea and Flood's generator as published; the value every
    reimplementation is checked against)."""
    assert inject.splitmix64(0, 0) == 0xE220A8397B1DCDAF
    # the counter form is the state sequence seed + k gamma: shifting the seed
    # by gamma shifts the counter by one
    for c in (0, 1, 17, 1 << 40):
        assert inject.splitmix64(12345 + inject.GAMMA, c) == inject.splitmix64(12345, c + 1)


def test_uniforms_and_irwin_hall():
    u = np.array([inject.uniform(99, inject.counter(3, i, d)) for i in range(500) for d in range(40)])
    assert u.min() >= 0.0 and u.max() < 1.0
    n = len(u)
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / n)
    assert abs(u.var() - 1 / 12) < 5 * 0.0745 / np.sqrt(n)  # sd of the sample variance of U(0,1)
    # 53-bit grid: every draw is an exact multiple of 2^-53
    assert np.all(np.floor(u * 2.0 ** 53) == u * 2.0 ** 53)


def _tube(order=1, n_particles=600, nz=10):
    cfg = workloads.make_config(1, n_particles=n_particles, walls="beam", tube=(8, 4, nz))
    return cfg


def test_injection_points_lie_on_injection_faces_by_area():
    cfg = _tube()
    t = topology.Topology(cfg["xyz"], cfg["tets"], 1, cfg["bface_tag"])
    g, c, vol = geometry.barycentric_maps(t.xyz, t.tets)
    table = inject.face_table(t)
    verts, owner, cum = table
    assert len(owner) == int(t.inject_face.sum()) > 0 and np.all(owner >= 0)
    # running areas against the faces' areas computed by the determinant rule
    area = np.array([0.5 * np.linalg.norm(np.cross(b - a, cc - a)) for a, b, cc in verts])
    assert np.allclose(np.diff(np.concatenate([[0.0], cum])), area, rtol=1e-13)
    hits = np.zeros(len(owner))
    faces = np.nonzero(t.inject_face & t.boundary_face)[0]
    drift, sigma = np.array([0.0, 0.0, 3e7]), np.array([3e5, 3e5, 3e5])
    vs = []
    for pid in range(3000):
        x, v, tt = inject.sample(table, 7, 5, pid, drift, sigma)
        lam = geometry.lam(g[tt][None], c[tt][None], x[None])[0]
        assert lam.min() > -1e-14 and np.sort(np.abs(lam))[0] < 1e-14   # on a face of its tet
        assert abs(x[2]) < 1e-15                                       # on z = 0
        f = t.tet_faces[tt, int(np.argmin(np.abs(lam)))]
        hits[int(np.nonzero(faces == f)[0][0])] += 1
        vs.append(v)
    # area-proportional face choice (chi-square, 5 sigma over the dof count)
    expect = 3000 * area / area.sum()
    chi2 = ((hits - expect) ** 2 / expect).sum()
    dof = len(area) - 1
    assert chi2 < dof + 5 * np.sqrt(2 * dof)
    vs = np.array(vs)
    assert np.all(np.abs(vs - drift) <= 6 * sigma + 1e-9)              # Irwin-Hall support
    assert np.allclose(vs.mean(axis=0), drift, atol=5 * 3e5 / np.sqrt(3000))
    assert np.allclose(vs.std(axis=0), sigma, rtol=0.1)


def test_absorbed_path_ends_on_the_wall_with_the_truncated_current():
    """A chord through an absorbing wall ends at the line-plane hit point, and
    its current equals that of the chord stopped at that point."""
    cfg = _tube(order=2)
    t = topology.Topology(cfg["xyz"], cfg["tets"], 2, cfg["bface_tag"])
    g, c, vol = geometry.barycentric_maps(t.xyz, t.tets)
    rng = np.random.default_rng(4)
    n = 50
    x0 = np.stack([rng.uniform(-0.003, 0.003, n), rng.uniform(-0.003, 0.003, n), rng.uniform(0.095, 0.099, n)], 1)
    own = np.array([int(np.argmax(geometry.lam(g, c, np.broadcast_to(p, (len(g), 3))).min(axis=1))) for p in x0])
    d = np.stack([rng.uniform(-1e-3, 1e-3, n), rng.uniform(-1e-3, 1e-3, n), np.full(n, 0.01)], 1)
    x1 = x0 + d
    v = d / 1e-9
    xe, ve, te, dg, nc, hs, st, ab = particles.walk_deposit(t, g, c, x0, x1, v, own, 1.0, t.n1,
                                                            absorb=t.tet_absorb)
    assert ab.all() and not st.any()
    s_hit = (0.10 - x0[:, 2]) / d[:, 2]
    assert np.allclose(xe, x0 + s_hit[:, None] * d, rtol=0, atol=1e-15)
    assert np.array_equal(ve, v)
    # the same chords stopped at the hit point, without absorbing walls
    xe2, _, te2, dg2, _, _, st2, ab2 = particles.walk_deposit(t, g, c, x0, xe, v, own, 1.0, t.n1)
    assert not ab2.any()
    assert np.abs(dg - dg2).max() <= 1e-13 * np.abs(dg).max()
    assert np.array_equal(te, te2)


@pytest.mark.parametrize("order", [1, 2])
def test_beam_steps_conserve_charge_on_interior_nodes(order):
    """Several steps of the beam through a short tube (absorbed at z = L,
    re-injected at z = 0): continuity on interior W0 DOFs to 1e-13 every
    step, Gauss's law carried, the count of particles fixed, every absorbed
    particle re-injected on an injection face."""
    cfg = _tube(n_particles=400, nz=4)
    cfg["dt"] = 1e-10  # 3 mm per step: a tenth of the particles leave in 4 steps
    o = osim.Sim(cfg["xyz"], cfg["tets"], order, cfg["q"], cfg["m"], cfg["weight"], cfg["B0"],
                 cfg["rho_ion"], bface_tag=cfg["bface_tag"])
    o.set_particles(cfg["x"], cfg["v"], cfg["tet"])
    o.set_injection(cfg["injectors"], cfg["inject_seed"])
    o.electrostatic_init()
    t = o.topo
    n_abs = 0
    for k in range(6):
        w = o.step(cfg["dt"])
        ab = w["absorbed"]
        n_abs += int(ab.sum())
        cont = w["continuity"][t.interior0]
        assert np.linalg.norm(cont) <= 1e-13 * np.linalg.norm(w["drho"][t.interior0])
        assert len(o.x) == 400
        if ab.any():
            assert np.all(np.abs(o.x[ab, 2]) < 1e-15)
        g = o.gauss_residual()[t.interior0]
        assert np.linalg.norm(g) <= 1e-9 * np.linalg.norm(o.rho[t.interior0])
    assert n_abs > 10


def test_absorbing_walls_need_injectors():
    cfg = _tube(n_particles=200, nz=2)
    cfg["dt"] = 3e-10
    o = osim.Sim(cfg["xyz"], cfg["tets"], 1, cfg["q"], cfg["m"], cfg["weight"], cfg["B0"],
                 cfg["rho_ion"], bface_tag=cfg["bface_tag"], matrices=False)
    o.set_particles(cfg["x"], cfg["v"], cfg["tet"])
    with pytest.raises(ValueError):  # 9 mm per step in a 10 cm tube: some reach z = L
        o.push_walk(cfg["dt"])


def test_two_species_reinjected_with_their_own_injectors():
    """Electrons and ions through the beam walls: each absorbed particle
    comes back with its own species' drift (ions slower, electrons faster),
    the slot keeps its species, and interior charge is conserved."""
    cfg = _tube(n_particles=300, nz=4)
    cfg["dt"] = 1e-10
    rng = np.random.default_rng(17)
    xi, ti = workloads.sample_uniform_in_tets(cfg["xyz"], cfg["tets"], 200, rng,
                                              subset=np.nonzero(cfg["xyz"][cfg["tets"]][:, :, 2].mean(axis=1) > 0.09)[0])
    vi = workloads.maxwellian(200, 1e4, rng, drift=(0.0, 0.0, 6e7))
    sp = [dict(q=-1.602176634e-19, m=9.1093837015e-31, weight=1.0, x=cfg["x"], v=cfg["v"], tet=cfg["tet"]),
          dict(q=1.602176634e-19, m=1.67262192e-27, weight=1.0, x=xi, v=vi, tet=ti)]
    o = osim.Sim(cfg["xyz"], cfg["tets"], 1, sp[0]["q"], sp[0]["m"], 1.0, cfg["B0"], 0.0,
                 bface_tag=cfg["bface_tag"])
    o.set_species(sp)
    o.set_injection([dict(species=0, v_drift=(0.0, 0.0, 3e7), v_sigma=(3e5,) * 3),
                     dict(species=1, v_drift=(0.0, 0.0, 1e5), v_sigma=(1e3,) * 3)], 99)
    t = o.topo
    seen = [0, 0]
    for _ in range(4):
        w = o.step(cfg["dt"])
        ab = w["absorbed"]
        for k, sl in enumerate((slice(0, 300), slice(300, 500))):
            idx = np.nonzero(ab[sl])[0] + sl.start
            seen[k] += len(idx)
            if len(idx):
                vz = o.v[idx, 2]
                want = 3e7 if k == 0 else 1e5
                assert np.all(np.abs(vz - want) <= 6 * (3e5 if k == 0 else 1e3) + 1e-6)
        cont = w["continuity"][t.interior0]
        assert np.linalg.norm(cont) <= 1e-13 * np.linalg.norm(w["drho"][t.interior0])
    assert seen[0] > 0 and seen[1] > 50   # ions start near z = L and drift out fast


def test_tube_wall_tags_mark_the_ends():
    """The workload's tags: every face on z = L absorbs (8 azimuthal x 4
    radial cells: 8 core triangles + 2 per ring quad = 56), the z = 0 faces
    inside half the radius inject (24), and all tagged faces are walls."""
    cfg = _tube(n_particles=10, nz=3)
    t = topology.Topology(cfg["xyz"], cfg["tets"], 1, cfg["bface_tag"])
    assert int(t.absorb_face.sum()) == 56 and int(t.inject_face.sum()) == 24
    assert np.all(t.boundary_face[t.absorb_face | t.inject_face])
    z = t.xyz[t.faces][:, :, 2]
    assert np.all(np.abs(z[t.absorb_face] - 0.10) < 1e-12) and np.all(np.abs(z[t.inject_face]) < 1e-12)
    assert not np.any(t.absorb_face & t.inject_face)

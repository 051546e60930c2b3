"""GPU parity of the absorbing and injecting particle walls against the
oracle, through the C ABI: the beam through a short tube (absorbed on z = L,
re-injected on the z = 0 faces inside the beam radius).

Every step starts both sides from the oracle's fields, so the particle half
of the step is compared on its own over several steps with absorptions and
re-injections: in the strict mode positions, velocities, owning tets,
crossing counts and hashes bit-exact (the re-injection draws from the same
counter-based generator and rounds every operation once on both sides),
Delta g and rho rel 1e-12, the absorbed count equal, continuity 1e-12 on the
device; in the contracted FP64 mode positions and velocities rel 1e-12.
"""

import numpy as np
import pytest

import workloads
from oracle import sim as osim
from gpu_helpers import assert_elementwise, build_lib, rel, assert_rho

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    return build_lib()


def _cfg(n=1001):
    cfg = workloads.make_config(1, n_particles=n, walls="beam", tube=(8, 4, 4))
    cfg["dt"] = 1e-10  # 3 mm per step in a 10 cm tube
    return cfg


def _pair(cfg, order, precision):
    from paper_2111_12411_gb300 import Simulation
    o = osim.Sim(cfg["xyz"], cfg["tets"], order, cfg["q"], cfg["m"], cfg["weight"], cfg["B0"], cfg["rho_ion"],
                 bface_tag=cfg["bface_tag"])
    o.set_particles(cfg["x"], cfg["v"], cfg["tet"])
    o.set_injection(cfg["injectors"], cfg["inject_seed"])
    o.electrostatic_init()
    c = dict(cfg, order=order)
    g = Simulation.from_config(c, precision=precision, es_init=False, diagnostics=True)
    return o, g


@pytest.mark.parametrize("order", [1, 2, 3])
@pytest.mark.parametrize("precision", ["fp64_strict", "fp64"])
def test_beam_walls_match_oracle(order, precision):
    cfg = _cfg()
    o, g = _pair(cfg, order, precision)
    assert g.info.n_absorb_faces == 56 and g.info.n_inject_faces == 24
    total = 0
    for k in range(5):
        g.set("E", o.e)
        g.set("E_PREV", o.e_prev)
        g.set("B", o.b)
        w = o.step(cfg["dt"])
        g.step(cfg["dt"])
        d = g.diag()
        assert d["absorbed"] == int(w["absorbed"].sum())
        total += d["absorbed"]
        xg, vg = g.get("X"), g.get("V")
        if precision == "fp64_strict":
            assert np.array_equal(xg, w["x"]) and np.array_equal(vg, w["v"])
            assert np.array_equal(g.get("TET"), w["tet"])
            assert np.array_equal(g.get("NCROSS"), w["ncross"])
            assert np.array_equal(g.get("HASH"), w["hash"])
        else:
            assert rel(xg, w["x"]) < 1e-12 and rel(vg, w["v"]) < 1e-12
        assert_elementwise(g.get("DG"), w["dg"], w["dg_abs"], 1e-12 if precision == "fp64_strict" else 1e-11,
                           "dg")
        assert_rho(g.get("RHO"), o, precision, "rho", g.get("X"), g.get("TET"))
        assert d["continuity_abs"] <= 1e-12 * d["continuity_ref"]
    assert total >= 20
    g.close()


def test_mixed_precision_walls_conserve_charge():
    cfg = _cfg(4001)
    from paper_2111_12411_gb300 import Simulation
    g = Simulation.from_config(dict(cfg, order=2), precision="mixed", diagnostics=True)
    n = 0
    for _ in range(6):
        g.step(cfg["dt"])
        d = g.diag()
        n += d["absorbed"]
        assert d["continuity_abs"] <= 1e-12 * d["continuity_ref"]
    x = g.get("X")
    assert n > 50 and np.all((x[:, 2] >= -1e-15) & (x[:, 2] <= 0.1 + 1e-15))
    assert g.n_particles == 4001
    g.close()


def test_wall_errors():
    from paper_2111_12411_gb300 import Batch, FemPICError, Simulation, native
    cfg = _cfg(300)
    g = Simulation(cfg["xyz"], cfg["tets"], 1, cfg["q"], cfg["m"], cfg["weight"], cfg["x"], cfg["v"],
                   cfg["tet"], B0=cfg["B0"], bface_tag=cfg["bface_tag"], es_init=False)
    with pytest.raises(FemPICError) as ei:  # absorbing faces and no injector
        g.step(cfg["dt"])
    assert ei.value.code == native.FEMPIC_ERR_STATE
    with pytest.raises(FemPICError) as ei:
        g.set_injection([dict(species=1, v_drift=(0, 0, 1), v_sigma=(0, 0, 0))], 1)
    assert ei.value.code == native.FEMPIC_ERR_ARG
    g.set_injection(cfg["injectors"], 5)
    vbad = g.get("V")
    vbad[7, 2] = np.inf
    with pytest.raises(FemPICError) as ei:  # refused on the host before any copy
        g.set("V", vbad)
    assert ei.value.code == native.FEMPIC_ERR_ARG
    g.step(cfg["dt"])
    with pytest.raises(FemPICError):
        Batch([g])
    g.close()
    with pytest.raises(FemPICError) as ei:
        Simulation(cfg["xyz"], cfg["tets"], 1, cfg["q"], cfg["m"], cfg["weight"], cfg["x"], cfg["v"],
                   cfg["tet"], bface_tag=cfg["bface_tag"], push="ab4")
    assert ei.value.code == native.FEMPIC_ERR_ARG


def test_two_species_walls_match_oracle():
    """Electrons and ions through the beam walls, each species re-injected by
    its own injector: strict mode bit-exact against the oracle over four
    steps (fields taken from the oracle every step)."""
    from paper_2111_12411_gb300 import Simulation
    cfg = workloads.make_config(1, n_particles=300, walls="beam", tube=(8, 4, 4))
    cfg["dt"] = 1e-10
    rng = np.random.default_rng(17)
    near_end = np.nonzero(cfg["xyz"][cfg["tets"]][:, :, 2].mean(axis=1) > 0.09)[0]
    xi, ti = workloads.sample_uniform_in_tets(cfg["xyz"], cfg["tets"], 200, rng, subset=near_end)
    vi = workloads.maxwellian(200, 1e4, rng, drift=(0.0, 0.0, 6e7))
    sp = [dict(q=-1.602176634e-19, m=9.1093837015e-31, weight=1.0, x=cfg["x"], v=cfg["v"], tet=cfg["tet"]),
          dict(q=1.602176634e-19, m=1.67262192e-27, weight=1.0, x=xi, v=vi, tet=ti)]
    inj = [dict(species=0, v_drift=(0.0, 0.0, 3e7), v_sigma=(3e5,) * 3),
           dict(species=1, v_drift=(0.0, 0.0, 1e5), v_sigma=(1e3,) * 3)]
    o = osim.Sim(cfg["xyz"], cfg["tets"], 1, sp[0]["q"], sp[0]["m"], 1.0, cfg["B0"], 0.0,
                 bface_tag=cfg["bface_tag"])
    o.set_species(sp)
    o.set_injection(inj, 99)
    g = Simulation(cfg["xyz"], cfg["tets"], 1, sp[0]["q"], sp[0]["m"], 1.0, cfg["x"], cfg["v"], cfg["tet"],
                   precision="fp64_strict", B0=cfg["B0"], es_init=False, diagnostics=True, species=sp,
                   bface_tag=cfg["bface_tag"])
    g.set_injection(inj, 99)
    total = 0
    for _ in range(4):
        g.set("E", o.e)
        g.set("E_PREV", o.e_prev)
        g.set("B", o.b)
        w = o.step(cfg["dt"])
        g.step(cfg["dt"])
        assert g.diag()["absorbed"] == int(w["absorbed"].sum())
        total += int(w["absorbed"].sum())
        assert np.array_equal(g.get("X"), w["x"]) and np.array_equal(g.get("V"), w["v"])
        assert np.array_equal(g.get("TET"), w["tet"]) and np.array_equal(g.get("HASH"), w["hash"])
        assert_rho(g.get("RHO"), o, "fp64_strict")
    assert total > 50
    g.close()


@pytest.mark.parametrize("precision", ["fp64_strict", "fp64"])
def test_full_size_beam_sampled(precision):
    """The benchmark's launch configuration: the drift tube at full size
    (132,480 tets, p = 2, 10^6 particles) with the beam absorbed at z = L and
    re-injected at z = 0.  One step from a seeded random field; 300 random
    particles and 200 whose straight path leaves through z = L are recomputed
    one by one by the oracle: the ones that stay against the walk (strict:
    bit-exact; contracted FP64: rel 1e-12), the absorbed ones against a fresh
    sample of the injector for their particle id at step 0 (bit-exact in both
    modes: the re-injection rounds every operation once).  Charge is
    conserved over all particles."""
    from paper_2111_12411_gb300 import Simulation
    from oracle import geometry, inject, particles as opart, topology as otopo
    from gpu_helpers import random_state
    cfg = workloads.make_config(1, walls="beam")
    g = Simulation.from_config(cfg, precision=precision, diagnostics=True, es_init=False)
    t = otopo.Topology(cfg["xyz"], cfg["tets"], 2, cfg["bface_tag"])
    rng = np.random.default_rng(6)
    e, b = random_state(t, rng, e_scale=1e4, b_scale=1e-3)
    g.set("E", e)
    g.set("E_PREV", e)
    g.set("B", b)
    g.step(cfg["dt"])
    d = g.diag()
    assert d["continuity_abs"] <= 1e-12 * d["continuity_ref"]
    assert d["absorbed"] > 1000
    z1 = cfg["x"][:, 2] + cfg["dt"] * cfg["v"][:, 2]
    leaving = np.nonzero(z1 > 0.1 + 1e-5)[0]
    idx = np.unique(np.concatenate([rng.choice(len(cfg["x"]), 300, replace=False),
                                    rng.choice(leaving, 200, replace=False)]))
    gg, cc, _ = geometry.barycentric_maps(t.xyz, t.tets)
    x0, v0, t0 = cfg["x"][idx], cfg["v"][idx], cfg["tet"][idx]
    E, B = opart.gather(t, gg, cc, e, b, cfg["B0"], x0, t0)
    vn = opart.boris(v0, E, B, cfg["q"], cfg["m"], cfg["dt"])
    x1 = x0 + cfg["dt"] * vn
    xe, ve, te, _, _, hs, _, ab = opart.walk_deposit(t, gg, cc, x0, x1, vn, t0, cfg["q"] * cfg["weight"], t.n1,
                                                     absorb=t.tet_absorb)
    assert ab.sum() >= 30
    table = inject.face_table(t)
    inj = cfg["injectors"][0]
    for i in np.nonzero(ab)[0]:
        xe[i], ve[i], te[i] = inject.sample(table, cfg["inject_seed"], 0, int(idx[i]), np.array(inj["v_drift"]),
                                            np.array(inj["v_sigma"]))
    xg, vg, tg = g.get("X")[idx], g.get("V")[idx], g.get("TET")[idx]
    assert np.array_equal(xg[ab], xe[ab]) and np.array_equal(vg[ab], ve[ab]) and np.array_equal(tg[ab], te[ab])
    k = ~ab
    if precision == "fp64_strict":
        assert np.array_equal(xg[k], xe[k]) and np.array_equal(vg[k], ve[k]) and np.array_equal(tg[k], te[k])
        assert np.array_equal(g.get("HASH")[idx][k], hs[k])
    else:
        assert rel(xg[k], xe[k]) < 1e-12 and rel(vg[k], ve[k]) < 1e-12
        ok = geometry.lam(gg[te[k]], cc[te[k]], xe[k]).min(axis=1) > 1e-9
        assert ok.mean() > 0.99 and np.array_equal(tg[k][ok], te[k][ok])
    g.close()

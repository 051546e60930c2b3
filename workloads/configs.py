"""The five synthetic workloads (C1..C5) with their seeded inputs.

Every config is seeded with ``20211123 + index``.  Plasma density, macro
particle weight and time step follow one rule where the workload does not fix
them: the electron plasma frequency is chosen so that ``v_ref / h`` equals
``omega_pe`` (``h`` the mean cell spacing) and ``dt = 0.5 / omega_pe``, so a
particle at ``v_ref`` moves about half a cell per step.  The drift tube uses
the expanding-beam table's time step (33.3 ps) and a weight set by a 5 mA beam
current instead (Section IV-D, Table "Expanding Particle Beam Parameters").
"""

import math

import numpy as np

from .meshes import kuhn_box, polar_tube, tet_volumes, tube_wall_tags
from .particles import sample_uniform_in_tets, maxwellian

Q_E = 1.602176634e-19        # elementary charge [C]
M_E = 9.1093837015e-31       # electron mass [kg]
EPS0 = 8.8541878128e-12      # vacuum permittivity [F/m]

SEED0 = 20211123
CONFIG_NAMES = ("c1_box6_p1", "c2_tube_p2", "c3_box37_p2_mixed", "c4_batched", "c5_serving")


def _density_for(omega_pe):
    return omega_pe * omega_pe * EPS0 * M_E / (Q_E * Q_E)


def _box_instance(n, order, n_particles, vth, b0z, seed, jitter=0.1,
                  beams=0.0, precision="fp64", steps=100):
    rng = np.random.default_rng(seed)
    xyz, tets = kuhn_box(n, n, n, jitter=jitter, seed=seed)
    h = 1.0 / n
    v_ref = max(vth, beams)
    omega = v_ref / h
    n_e = _density_for(omega)
    x, owner = sample_uniform_in_tets(xyz, tets, n_particles, rng)
    v = maxwellian(n_particles, vth, rng)
    if beams > 0.0:
        half = n_particles // 2
        v[:half, 2] += beams
        v[half:, 2] -= beams
    volume = 1.0
    return dict(
        order=order, xyz=xyz, tets=tets, x=x, v=v, tet=owner,
        q=-Q_E, m=M_E, weight=n_e * volume / n_particles,
        dt=0.5 / omega, B0=(0.0, 0.0, b0z), rho_ion=Q_E * n_e,
        steps=steps, precision=precision)


def make_config(name_or_index, n_particles=None, steps=None, walls="reflect", tube=(24, 12, 80)):
    """Build one config; ``n_particles``/``steps`` override the sizes.

    Drift tube only: ``walls="beam"`` makes the beam flow through (particles
    absorbed on z = L and re-injected on the z = 0 faces inside the beam
    radius with the beam's velocity distribution, seed ``seed``); the default
    reflects at every wall.  ``tube`` = (azimuthal, radial, axial) cells."""
    idx = (CONFIG_NAMES.index(name_or_index) if isinstance(name_or_index, str)
           else int(name_or_index))
    seed = SEED0 + idx
    if idx == 0:
        cfg = _box_instance(6, 1, n_particles or 10_000, 1.0e6, 0.1, seed, steps=100)
    elif idx == 1:
        rng = np.random.default_rng(seed)
        xyz, tets = polar_tube(*tube, radius=0.01, length=0.10)
        n = n_particles or 1_000_000
        r_beam, v0, current = 0.005, 3.0e7, 5.0e-3
        cent = xyz[tets].mean(axis=1)
        core = np.nonzero(np.hypot(cent[:, 0], cent[:, 1]) < r_beam)[0]
        x, owner = sample_uniform_in_tets(xyz, tets, n, rng, subset=core)
        v = maxwellian(n, 0.01 * v0, rng, drift=(0.0, 0.0, v0))
        beam_volume = float(np.abs(tet_volumes(xyz, tets[core])).sum())
        n_e = current / (Q_E * v0 * math.pi * r_beam * r_beam)
        cfg = dict(order=2, xyz=xyz, tets=tets, x=x, v=v, tet=owner,
                   q=-Q_E, m=M_E, weight=n_e * beam_volume / n,
                   dt=33.3e-12, B0=(0.0, 0.0, 1.0), rho_ion=0.0,
                   steps=1000, precision="fp64")
        if walls == "beam":
            cfg["bface_tag"] = tube_wall_tags(xyz, tets, 0.10, r_beam)
            cfg["injectors"] = [dict(species=0, v_drift=(0.0, 0.0, v0), v_sigma=(0.01 * v0,) * 3)]
            cfg["inject_seed"] = seed
        elif walls != "reflect":
            raise ValueError(walls)
    elif idx == 2:
        cfg = _box_instance(37, 2, n_particles or 10_000_000, 1.0e6, 0.0, seed,
                            beams=2.0e7, precision="mixed", steps=500)
    elif idx in (3, 4):
        raise ValueError("use make_batch / make_requests for the batched and serving workloads")
    else:
        raise ValueError(name_or_index)
    if steps is not None:
        cfg["steps"] = steps
    cfg["name"] = CONFIG_NAMES[idx]
    cfg["seed"] = seed
    return cfg


def make_batch(n_instances=64, seed=SEED0 + 3, np_range=(1e4, 1e6),
               nt_range=(2e3, 5e4), steps=200, precision="mixed"):
    """The batched workload: independent box instances of mixed size/order."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_instances):
        nt = math.exp(rng.uniform(math.log(nt_range[0]), math.log(nt_range[1])))
        n = max(6, int(round((nt / 6.0) ** (1.0 / 3.0))))
        order = int(rng.integers(1, 3))
        npart = int(math.exp(rng.uniform(math.log(np_range[0]), math.log(np_range[1]))))
        b0z = float(rng.uniform(0.0, 1.0))
        cfg = _box_instance(n, order, npart, 1.0e6, b0z, int(rng.integers(1 << 31)),
                            precision=precision, steps=steps)
        cfg["name"] = f"batch{i}"
        out.append(cfg)
    return out


def make_requests(n_requests=512, rate_hz=50.0, seed=SEED0 + 4, max_particles=4e6,
                  chunk_steps=50, chunks=(1, 4)):
    """Serving workload: Poisson arrivals of box simulations (sizes only).

    Returns dicts with the arrival time and the instance parameters; the
    instance inputs are built lazily with ``build_request``.
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    for i in range(n_requests):
        t += rng.exponential(1.0 / rate_hz)
        nt = math.exp(rng.uniform(math.log(2e3), math.log(5e4)))
        n = max(6, int(round((nt / 6.0) ** (1.0 / 3.0))))
        reqs.append(dict(
            id=i, arrival=t, n=n, order=int(rng.integers(1, 3)),
            n_particles=int(math.exp(rng.uniform(math.log(1e4), math.log(max_particles)))),
            b0z=float(rng.uniform(0.0, 1.0)), seed=int(rng.integers(1 << 31)),
            chunk_steps=chunk_steps, n_chunks=int(rng.integers(chunks[0], chunks[1] + 1))))
    return reqs


def build_request(req, precision="mixed"):
    cfg = _box_instance(req["n"], req["order"], req["n_particles"], 1.0e6, req["b0z"],
                        req["seed"], precision=precision,
                        steps=req["chunk_steps"] * req["n_chunks"])
    cfg["name"] = f"req{req['id']}"
    return cfg


def random_dof_vector(n, scale, rng, zero_mask=None):
    """Random normal vector (a synthetic field state), zeros where masked."""
    v = rng.normal(0.0, scale, size=n)
    if zero_mask is not None:
        v[np.asarray(zero_mask, dtype=bool)] = 0.0
    return v

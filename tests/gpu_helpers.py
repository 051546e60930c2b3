"""Shared helpers of the GPU parity tests (the library and the oracle fed with
the same seeded inputs)."""

import numpy as np

import workloads
from oracle import sim as osim


def build_lib():
    from paper_2111_12411_gb300 import build
    build.build()
    from paper_2111_12411_gb300 import native
    native.load()
    return native


def random_state(topo, rng, e_scale=1e3, b_scale=1e-4):
    e = workloads.random_dof_vector(topo.n1, e_scale, rng, topo.pec1)
    b = workloads.random_dof_vector(topo.n2, b_scale, rng)
    return e, b


def pair(cfg, order=None, precision="fp64", matrices=True, **kw):
    """An oracle Sim and a library Simulation on the same config."""
    from paper_2111_12411_gb300 import Simulation
    order = order or cfg["order"]
    o = osim.Sim(cfg["xyz"], cfg["tets"], order, cfg["q"], cfg["m"], cfg["weight"], cfg["B0"],
                 cfg["rho_ion"], matrices=matrices)
    o.set_particles(cfg["x"], cfg["v"], cfg["tet"])
    g = Simulation(cfg["xyz"], cfg["tets"], order, cfg["q"], cfg["m"], cfg["weight"], cfg["x"],
                   cfg["v"], cfg["tet"], precision=precision, B0=cfg["B0"], rho_ion=cfg["rho_ion"], **kw)
    return o, g


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)

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


def assert_elementwise(a, b, scale, tol, what):
    """|a_k - b_k| <= tol * scale_k for every element k.

    For a deposited vector, scale_k is the oracle's sum of the absolute
    values of the terms added into element k (the size of its rounding error
    whatever the order of the sum), so a small element is held to its own
    terms and not to the vector's norm; an element with no terms must be
    exactly zero on both sides."""
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    err = np.abs(a - b)
    bound = tol * np.asarray(scale, dtype=np.float64)
    bad = np.nonzero(~(err <= bound))[0]
    assert bad.size == 0, (f"{what}: {bad.size} of {a.size} elements off; first {bad[:4].tolist()} "
                           f"err {err[bad[:4]].tolist()} bound {bound[bad[:4]].tolist()}")


def assert_close_to_scale(a, b, tol, what, floor=1e-3):
    """|a_k - b_k| <= tol * max(|b_k|, floor * max|b|) for every element:
    per-element relative error, with a floor for elements near zero."""
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    scale = np.maximum(np.abs(b), floor * (np.abs(b).max() if b.size else 0.0))
    assert_elementwise(a, b, scale, tol, what)


def assert_rho(g_rho, o, precision, what="rho", gx=None, gtet=None):
    """Charge per W0 DOF against the oracle.  Strict mode: the same end points
    and the same formulas, so 1e-12 of the sum of the terms' absolute values.
    A contracted kernel (fused multiply-adds) ends its particles within its
    position tolerance of the oracle's and evaluates W0 at barycentrics a few
    ulps apart: its charge is compared with the oracle's measurement at the
    device's own end points (gx, gtet), to 1e-12 of the terms plus 1e-14
    |q w| per contributing particle (an order-p Lagrange function amplifies
    an absolute difference in lambda by its derivative, at most ~2 p^2)."""
    if precision == "fp64_strict" or gx is None:
        scale = o.rho_abs if precision == "fp64_strict" else o.rho_abs + 1e-2 * o.rho_cnt
        assert_elementwise(g_rho, o.rho, scale, 1e-12, what)
        return
    keep = (o.rho_abs, o.rho_cnt)
    ref = o._measure_rho(np.asarray(gx, dtype=np.float64).reshape(-1, 3), np.asarray(gtet, dtype=np.int64))
    scale = o.rho_abs + 1e-2 * o.rho_cnt
    o.rho_abs, o.rho_cnt = keep
    assert_elementwise(g_rho, ref, scale, 1e-12, what)


def assert_particles_close(gx, gv, wx, wv, tol, extent, what=""):
    """Per particle: |x_g - x_o| <= tol * extent (a position's rounding scales
    with the chord and the domain, not with its own coordinates) and
    |v_g - v_o| <= tol * |v_o| (the particle's speed)."""
    dx = np.linalg.norm(np.asarray(gx) - wx, axis=1)
    dv = np.linalg.norm(np.asarray(gv) - wv, axis=1)
    sv = np.linalg.norm(wv, axis=1)
    bx = np.nonzero(~(dx <= tol * extent))[0]
    bv = np.nonzero(~(dv <= tol * sv))[0]
    assert bx.size == 0, f"x{what}: {bx.size} particles off, first {bx[:4].tolist()} |dx| {dx[bx[:4]].tolist()}"
    assert bv.size == 0, f"v{what}: {bv.size} particles off, first {bv[:4].tolist()} |dv|/|v| {(dv / sv)[bv[:4]].tolist()}"


def assert_solves_system(A, e, rhs, rhs_terms, rtol, what="e"):
    """||A e - rhs|| <= 10 rtol ||rhs|| + 256 eps ||rhs_terms||: the device
    solved its own right-hand side to rtol, which differs from the oracle's by
    the rounding of the terms that make it up (rhs_terms: the sum of their
    absolute values per row; they cancel when e is a gradient field)."""
    eps = np.finfo(np.float64).eps
    res = np.linalg.norm(A @ e - rhs)
    bound = 10 * rtol * np.linalg.norm(rhs) + 256 * eps * np.linalg.norm(rhs_terms)
    assert res <= bound, f"{what}: residual {res:.3e} > bound {bound:.3e}"

"""Interpolatory Whitney bases of order 1 and 2 on a tetrahedron (Appendix);
order 3 is delegated to ``basis3``.

The Appendix builds each basis as an interpolatory Silvester polynomial
(P_i, shifted P^_i) times a lowest-order Whitney form.  Readings taken here
(the printed formulas are ambiguous or garbled, see the design notes):

* W1 of order p uses multi-indices (a,b,c,d) with a,b >= 1 on the edge's own
  vertices and a+b+c+d = p+1, with the Silvester scale equal to p+1.  At p=2
  this gives, per edge (s<t), (3 l_s - 1) w_st and (3 l_t - 1) w_st, and per
  face (s<t<u) the three candidates 3 l_u w_st, 3 l_t w_su, 3 l_s w_tu which
  obey l_u w_st - l_t w_su + l_s w_tu = 0; the last is dropped.  20 functions.
* W2 of order p uses (a,b,c,d) with a,b,c >= 1 on the face's vertices,
  a+b+c+d = p+2, scale p+2, on the Whitney face form
  w_stu = 2 (l_s grad l_t x grad l_u + l_t grad l_u x grad l_s
  + l_u grad l_s x grad l_t) (the printed middle term is a typo).  At p=2:
  (4 l_x - 1) w_stu for x in {s,t,u} per face and the interior candidates
  4 l_i w_(face opposite i), i = 0..3, with one dependency; the one for i=3
  is dropped.  15 functions.
* W0 of order p is the Lagrange basis on the lattice points (the printed
  l_s P^ P P P form equals it up to a constant factor per function).

``lam`` has shape [..., 4], ``g`` (the barycentric gradients) [..., 4, 3].
All arithmetic is written in a fixed order, one rounding per operation.

Test infrastructure only: part of the CPU oracle, which the product library
never imports.
"""

import numpy as np

from . import basis3
from .geometry import cross
from .topology import LOCAL_EDGES, LOCAL_FACES


def n_local(order):
    """(n0, n1, n2) local DOF counts (Appendix: (k+1)(k+2)(k+3)/6,
    k(k+2)(k+3)/2, k(k+1)(k+3)/2)."""
    k = order
    return (k + 1) * (k + 2) * (k + 3) // 6, k * (k + 2) * (k + 3) // 2, k * (k + 1) * (k + 3) // 2


def w1_spec(order):
    """For each local W1 function: (a, b, mult_vertex, mult_kind).

    The function is m(l) * (l_a grad l_b - l_b grad l_a) with
    m = 3 l_x - 1 (kind 'e'), m = 3 l_x (kind 'f') or m = 1 (order 1).
    """
    if order == 1:
        return [(s, t, -1, "1") for (s, t) in LOCAL_EDGES]
    spec = []
    for (s, t) in LOCAL_EDGES:
        spec.append((s, t, s, "e"))
        spec.append((s, t, t, "e"))
    for (s, t, u) in LOCAL_FACES:
        spec.append((s, t, u, "f"))
        spec.append((s, u, t, "f"))
    return spec


def w2_spec(order):
    """For each local W2 function: (face_index, mult_vertex, mult_kind).

    The function is m(l) * w_face with m = 4 l_x - 1 ('e'), 4 l_x ('i') or 1.
    """
    if order == 1:
        return [(f, -1, "1") for f in range(4)]
    spec = []
    for f, verts in enumerate(LOCAL_FACES):
        for x in verts:
            spec.append((f, x, "e"))
    for i in range(3):
        spec.append((i, i, "i"))
    return spec


def _mult1(kind, lx):
    if kind == "1":
        return None
    if kind == "e":
        return 3.0 * lx - 1.0
    return 3.0 * lx


def whitney_edge(lam, g, a, b):
    """w_ab = l_a grad l_b - l_b grad l_a."""
    return lam[..., a, None] * g[..., b, :] - lam[..., b, None] * g[..., a, :]


def whitney_face(lam, g, f):
    """w_stu for local face f = (s,t,u)."""
    s, t, u = LOCAL_FACES[f]
    x_tu = cross(g[..., t, :], g[..., u, :])
    x_us = cross(g[..., u, :], g[..., s, :])
    x_st = cross(g[..., s, :], g[..., t, :])
    return ((lam[..., s, None] * x_tu + lam[..., t, None] * x_us)
            + lam[..., u, None] * x_st) * 2.0


def w1(order, lam, g):
    if order == 3:
        return basis3.w1(lam, g)
    out = []
    for (a, b, x, kind) in w1_spec(order):
        w = whitney_edge(lam, g, a, b)
        m = _mult1(kind, lam[..., x]) if x >= 0 else None
        out.append(w if m is None else m[..., None] * w)
    return np.stack(out, axis=-2)


def curl_w1(order, lam, g):
    """curl(m w_ab) = grad m x w_ab + 2 m grad l_a x grad l_b."""
    if order == 3:
        return basis3.curl_w1(lam, g)
    out = []
    for (a, b, x, kind) in w1_spec(order):
        c = cross(g[..., a, :], g[..., b, :]) * 2.0
        if kind == "1":
            out.append(c)
            continue
        m = _mult1(kind, lam[..., x])
        gm = g[..., x, :] * 3.0
        out.append(cross(gm, whitney_edge(lam, g, a, b)) + m[..., None] * c)
    return np.stack(out, axis=-2)


def w2(order, lam, g):
    if order == 3:
        return basis3.w2(lam, g)
    out = []
    for (f, x, kind) in w2_spec(order):
        w = whitney_face(lam, g, f)
        if kind == "1":
            out.append(w)
        elif kind == "e":
            out.append((4.0 * lam[..., x] - 1.0)[..., None] * w)
        else:
            out.append((4.0 * lam[..., x])[..., None] * w)
    return np.stack(out, axis=-2)


def div_w2(order, lam, g):
    """div(m w_f) = grad m . w_f + m div w_f, div w_stu = 6 grad l_s . (grad l_t x grad l_u)."""
    if order == 3:
        return basis3.div_w2(lam, g)
    out = []
    for (f, x, kind) in w2_spec(order):
        s, t, u = LOCAL_FACES[f]
        dv = 6.0 * np.einsum("...k,...k->...", g[..., s, :], cross(g[..., t, :], g[..., u, :]))
        if kind == "1":
            out.append(dv)
            continue
        w = whitney_face(lam, g, f)
        gm = g[..., x, :] * 4.0
        m = 4.0 * lam[..., x] - (1.0 if kind == "e" else 0.0)
        out.append(np.einsum("...k,...k->...", gm, w) + m * dv)
    return np.stack(out, axis=-1)


def w0(order, lam):
    if order == 3:
        return basis3.w0(lam)
    if order == 1:
        return lam.copy()
    vals = [lam[..., s] * (2.0 * lam[..., s] - 1.0) for s in range(4)]
    vals += [(4.0 * lam[..., s]) * lam[..., t] for (s, t) in LOCAL_EDGES]
    return np.stack(vals, axis=-1)


def grad_w0(order, lam, g):
    if order == 3:
        return basis3.grad_w0(lam, g)
    if order == 1:
        return g.copy() * np.ones(lam.shape + (1,))
    vals = [(4.0 * lam[..., s] - 1.0)[..., None] * g[..., s, :] for s in range(4)]
    vals += [(lam[..., t, None] * g[..., s, :] + lam[..., s, None] * g[..., t, :]) * 4.0
             for (s, t) in LOCAL_EDGES]
    return np.stack(vals, axis=-2)


def combine(coef, vals):
    """sum_j coef[..., j] * vals[..., j, :] accumulated in j order."""
    acc = np.zeros(vals.shape[:-2] + (vals.shape[-1],))
    for j in range(vals.shape[-2]):
        acc = acc + coef[..., j, None] * vals[..., j, :]
    return acc

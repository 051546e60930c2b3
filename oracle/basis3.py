"""Interpolatory bases of order 3 (Appendix), built from their general form.

The Appendix writes every basis function as a product of Silvester
polynomials in the barycentric coordinates times a lowest-order Whitney form:

  P_i(l) = prod_{m=0}^{i-1} (n l - m) / i!  (P_0 = 1),
  P^_i(l) = prod_{m=1}^{i-1} (n l - m) / (i-1)!  (P^_1 = 1),

with the scale n read as the multi-index sum (the same reading as at orders
1 and 2).  At order p = 3:

* W0 (20): P_a(l_0) P_b(l_1) P_c(l_2) P_d(l_3), a+b+c+d = 3, scale 3, the
  Lagrange basis on the lattice; numbered nodes, then 2 per edge (the lattice
  point nearer the lower vertex first), then 1 per face.
* W1 (45): m(l) w_st with m = P^_a(l_s) P^_b(l_t) P_c(l_u) P_d(l_v), a, b >= 1,
  a+b+c+d = 4, scale 4.  Per edge (c = d = 0): (a, b) = (3,1), (2,2), (1,3).
  Per face s<t<u (d = 0, c >= 1): the candidates of the pairs (s,t) and (s,u)
  with (a, b, c) = (2,1,1), (1,2,1), (1,1,2) (a on the pair's first vertex, b
  on its second, c on the face's third); the pair (t,u), whose edge avoids
  the face's lowest vertex, is dropped (l_s w_tu = l_t w_su - l_u w_st, as at
  order 2).  Interior (all four indices 1): the pairs (0,1), (0,2), (0,3);
  the other three are combinations of these (one relation l_x (l_u w_st -
  l_t w_su + l_s w_tu) = 0 per face).  6*3 + 4*6 + 3 = 45.
* W2 (36): m(l) w_stu with m = P^_a(l_s) P^_b(l_t) P^_c(l_u) P_d(l_v), a, b,
  c >= 1, a+b+c+d = 5, scale 5.  Per face (d = 0): (a, b, c) = (3,1,1),
  (1,3,1), (1,1,3), (2,2,1), (2,1,2), (1,2,2).  Interior (d >= 1): the faces
  opposite vertices 0, 1, 2 with (a, b, c, d) = (2,1,1,1), (1,2,1,1),
  (1,1,2,1), (1,1,1,2); the face opposite vertex 3 is dropped
  (sum_i (-1)^i l_i w_(opp i) = 0 times the linear multipliers).
  4*6 + 12 = 36.

Global numbering (Topology): W1 edges 3*edge + v, faces 3*N_e + 6*face + v,
interior 3*N_e + 6*N_f + 3*tet + v; W2 faces 6*face + v, interior
6*N_f + 12*tet + v.

Values and derivatives of the multipliers are formed by the product rule.

Test infrastructure only: part of the CPU oracle, which the product library
never imports.
"""

from math import factorial

import numpy as np

from .geometry import cross

LOCAL_EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))
LOCAL_FACES = ((1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2))


def silvester(i, n, lam):
    """P_i(l) and dP_i/dl at scale n."""
    val = np.ones_like(lam)
    der = np.zeros_like(lam)
    for m in range(i):
        f = n * lam - m
        der = der * f + val * n
        val = val * f
    return val / factorial(i), der / factorial(i)


def silvester_hat(i, n, lam):
    """P^_i(l) and its derivative at scale n."""
    val = np.ones_like(lam)
    der = np.zeros_like(lam)
    for m in range(1, i):
        f = n * lam - m
        der = der * f + val * n
        val = val * f
    return val / factorial(i - 1), der / factorial(i - 1)


def _other(s, t):
    return tuple(k for k in range(4) if k not in (s, t))


def w1_spec3():
    """(a, b, {vertex: (index, hat)}) for the 45 local W1 functions."""
    spec = []
    for (s, t) in LOCAL_EDGES:
        for (ia, ib) in ((3, 1), (2, 2), (1, 3)):
            spec.append((s, t, {s: (ia, True), t: (ib, True)}))
    for (s, t, u) in LOCAL_FACES:
        for (p, q, r) in ((s, t, u), (s, u, t)):
            for (ia, ib, ic) in ((2, 1, 1), (1, 2, 1), (1, 1, 2)):
                spec.append((p, q, {p: (ia, True), q: (ib, True), r: (ic, False)}))
    for (s, t) in ((0, 1), (0, 2), (0, 3)):
        u, v = _other(s, t)
        spec.append((s, t, {s: (1, True), t: (1, True), u: (1, False), v: (1, False)}))
    return spec


def w2_spec3():
    """(face, {vertex: (index, hat)}) for the 36 local W2 functions."""
    spec = []
    for f, (s, t, u) in enumerate(LOCAL_FACES):
        for (ia, ib, ic) in ((3, 1, 1), (1, 3, 1), (1, 1, 3), (2, 2, 1), (2, 1, 2), (1, 2, 2)):
            spec.append((f, {s: (ia, True), t: (ib, True), u: (ic, True)}))
    for f in (0, 1, 2):
        s, t, u = LOCAL_FACES[f]
        for (ia, ib, ic, idd) in ((2, 1, 1, 1), (1, 2, 1, 1), (1, 1, 2, 1), (1, 1, 1, 2)):
            spec.append((f, {s: (ia, True), t: (ib, True), u: (ic, True), f: (idd, False)}))
    return spec


def w0_spec3():
    """Lattice multi-indices (a, b, c, d), a+b+c+d = 3, in the global order."""
    spec = [tuple(3 if k == v else 0 for k in range(4)) for v in range(4)]
    for (s, t) in LOCAL_EDGES:
        for (ia, ib) in ((2, 1), (1, 2)):
            spec.append(tuple(ia if k == s else (ib if k == t else 0) for k in range(4)))
    for (s, t, u) in LOCAL_FACES:
        spec.append(tuple(1 if k in (s, t, u) else 0 for k in range(4)))
    return spec


def _multiplier(factors, scale, lam, g):
    """m(l) and grad m for m = prod over vertices of P or P^."""
    val = np.ones(lam.shape[:-1])
    dm = np.zeros(lam.shape[:-1] + (4,))
    for v, (i, hat) in factors.items():
        pv, dv = (silvester_hat if hat else silvester)(i, scale, lam[..., v])
        dm = dm * pv[..., None]
        dm[..., v] = dm[..., v] + val * dv
        val = val * pv
    grad = np.einsum("...i,...ik->...k", dm, g)
    return val, grad


def whitney_edge(lam, g, a, b):
    return lam[..., a, None] * g[..., b, :] - lam[..., b, None] * g[..., a, :]


def whitney_face(lam, g, f):
    s, t, u = LOCAL_FACES[f]
    return ((lam[..., s, None] * cross(g[..., t, :], g[..., u, :])
             + lam[..., t, None] * cross(g[..., u, :], g[..., s, :]))
            + lam[..., u, None] * cross(g[..., s, :], g[..., t, :])) * 2.0


def w1(lam, g):
    out = []
    for (a, b, fac) in w1_spec3():
        m, _ = _multiplier(fac, 4, lam, g)
        out.append(m[..., None] * whitney_edge(lam, g, a, b))
    return np.stack(out, axis=-2)


def curl_w1(lam, g):
    """curl(m w_ab) = grad m x w_ab + 2 m grad l_a x grad l_b."""
    out = []
    for (a, b, fac) in w1_spec3():
        m, gm = _multiplier(fac, 4, lam, g)
        out.append(cross(gm, whitney_edge(lam, g, a, b)) + (2.0 * m)[..., None] * cross(g[..., a, :], g[..., b, :]))
    return np.stack(out, axis=-2)


def w2(lam, g):
    out = []
    for (f, fac) in w2_spec3():
        m, _ = _multiplier(fac, 5, lam, g)
        out.append(m[..., None] * whitney_face(lam, g, f))
    return np.stack(out, axis=-2)


def div_w2(lam, g):
    """div(m w_f) = grad m . w_f + m div w_f, div w_stu = 6 grad l_s . (grad l_t x grad l_u)."""
    out = []
    for (f, fac) in w2_spec3():
        s, t, u = LOCAL_FACES[f]
        m, gm = _multiplier(fac, 5, lam, g)
        dv = 6.0 * np.einsum("...k,...k->...", g[..., s, :], cross(g[..., t, :], g[..., u, :]))
        out.append(np.einsum("...k,...k->...", gm, whitney_face(lam, g, f)) + m * dv)
    return np.stack(out, axis=-1)


def w0(lam):
    out = []
    for idx in w0_spec3():
        m, _ = _multiplier({v: (i, False) for v, i in enumerate(idx)}, 3, lam,
                           np.zeros(lam.shape[:-1] + (4, 3)))
        out.append(m)
    return np.stack(out, axis=-1)


def grad_w0(lam, g):
    out = []
    for idx in w0_spec3():
        _, gm = _multiplier({v: (i, False) for v, i in enumerate(idx)}, 3, lam, g)
        out.append(gm)
    return np.stack(out, axis=-2)


def w1_along(lam, d):
    """W1_j . (b - a) on a straight chord: m_j(l) (l_a d_b - l_b d_a), where d
    [..., 4] are the barycentric increments lambda(b) - lambda(a)
    (grad l . (b - a) = d)."""
    out = []
    for (a, b, fac) in w1_spec3():
        m, _ = _multiplier(fac, 4, lam, np.zeros(lam.shape[:-1] + (4, 3)))
        out.append(m * (lam[..., a] * d[..., b] - lam[..., b] * d[..., a]))
    return np.stack(out, axis=-1)

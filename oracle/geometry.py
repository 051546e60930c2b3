"""Barycentric maps of the tets.

For a tet with (sorted) vertices P0..P3 the barycentric coordinates are affine,
lambda_i(x) = g_i . x + c_i.  With e_k = P_k - P0 and det = e1 . (e2 x e3):
g_1 = (e2 x e3)/det, g_2 = (e3 x e1)/det, g_3 = (e1 x e2)/det,
g_0 = -(g_1 + g_2 + g_3), c_i = -g_i . P0 (i >= 1), c_0 = 1 - (c_1 + c_2 + c_3).

Every operation is written out in a fixed order with one rounding per
operation (Python/numpy float64, no fused multiply-add), so that the walk's
decisions, which depend on the signs of lambda, are reproducible.

Test infrastructure only: part of the CPU oracle, which the product library
never imports.
"""

import numpy as np


def cross(a, b):
    """Componentwise cross product of [..., 3] arrays."""
    return np.stack([a[..., 1] * b[..., 2] - a[..., 2] * b[..., 1],
                     a[..., 2] * b[..., 0] - a[..., 0] * b[..., 2],
                     a[..., 0] * b[..., 1] - a[..., 1] * b[..., 0]], axis=-1)


def dot3(a, b):
    return (a[..., 0] * b[..., 0] + a[..., 1] * b[..., 1]) + a[..., 2] * b[..., 2]


def barycentric_maps(xyz, sorted_tets):
    """Return ``g`` [Nt,4,3], ``c`` [Nt,4] and the unsigned volume [Nt]."""
    p = xyz[sorted_tets]
    p0 = p[:, 0]
    e1, e2, e3 = p[:, 1] - p0, p[:, 2] - p0, p[:, 3] - p0
    n1, n2, n3 = cross(e2, e3), cross(e3, e1), cross(e1, e2)
    det = dot3(e1, n1)
    g = np.empty((len(p), 4, 3))
    g[:, 1] = n1 / det[:, None]
    g[:, 2] = n2 / det[:, None]
    g[:, 3] = n3 / det[:, None]
    g[:, 0] = -((g[:, 1] + g[:, 2]) + g[:, 3])
    c = np.empty((len(p), 4))
    for i in (1, 2, 3):
        c[:, i] = -dot3(g[:, i], p0)
    c[:, 0] = 1.0 - ((c[:, 1] + c[:, 2]) + c[:, 3])
    return g, c, np.abs(det) / 6.0


def lam(g, c, x):
    """lambda_i(x) = ((g_i0 x0 + g_i1 x1) + g_i2 x2) + c_i for [...,4,3], [...,4], [...,3]."""
    return ((g[..., 0] * x[..., None, 0] + g[..., 1] * x[..., None, 1])
            + g[..., 2] * x[..., None, 2]) + c

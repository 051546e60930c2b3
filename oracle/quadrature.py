"""Quadrature rules.

* ``gauss_legendre01(n)``: n-point Gauss-Legendre nodes/weights on [0, 1]
  (numpy's Legendre-Gauss rule, mapped), exact for degree 2n-1.
* ``tet_rule(n)``: a collapsed-cube (conical product) rule on the reference
  tet {x,y,z >= 0, x+y+z <= 1}: x = u, y = (1-u) v, z = (1-u)(1-v) w with
  Jacobian (1-u)^2 (1-v) and n Gauss-Legendre points per direction.  A
  polynomial of total degree d becomes degree d+2 in u, so the rule is exact
  for d <= 2n-3.  Returns barycentric points [Q,4] and weights summing to 1/6.
* ``tri_rule(n)``: the same construction on the reference triangle
  {x, y >= 0, x + y <= 1}: x = u, y = (1-u) v, Jacobian (1-u); exact for
  total degree d <= 2n-2.  Returns barycentric points [Q,3] and weights
  summing to 1/2.

Test infrastructure only: part of the CPU oracle, which the product library
never imports.
"""

import numpy as np


def gauss_legendre01(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def tet_rule(n):
    x, w = gauss_legendre01(n)
    pts, wts = [], []
    for iu, u in enumerate(x):
        for iv, v in enumerate(x):
            for iw, s in enumerate(x):
                px = u
                py = (1.0 - u) * v
                pz = (1.0 - u) * (1.0 - v) * s
                jac = (1.0 - u) ** 2 * (1.0 - v)
                pts.append((1.0 - px - py - pz, px, py, pz))
                wts.append(w[iu] * w[iv] * w[iw] * jac)
    return np.array(pts), np.array(wts)


def tri_rule(n):
    x, w = gauss_legendre01(n)
    pts, wts = [], []
    for iu, u in enumerate(x):
        for iv, v in enumerate(x):
            px = u
            py = (1.0 - u) * v
            pts.append((1.0 - px - py, px, py))
            wts.append(w[iu] * w[iv] * (1.0 - u))
    return np.array(pts), np.array(wts)

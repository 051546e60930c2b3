"""Divergence-free representation of an impressed magnetic flux density
(Section III-C, eq. conB).

The Galerkin projection [*mu^-1] b = f, f_i = <W2_i, B^i>, is divergence free
only when it reproduces B^i exactly.  The constrained form minimises the same
energy under Gauss's magnetic law:

  [ [*mu^-1]  [div]^T ] [ b      ]   [ f ]
  [ [div]     0       ] [ lambda ] = [ 0 ],   [div] = [*3]^-1 [~div],

with [*3]_ij = <W3_i, W3_j> and [~div]_ij = <W3_i, div W2_j> over the volume
functions W3 (Appendix).  Readings:

* W3 of order p: P^_a(l_0) P^_b(l_1) P^_c(l_2) P^_d(l_3), a, b, c, d >= 1,
  a+b+c+d = p+3, scale p+3 (the Appendix's Q3 with the scale read as the index
  sum), times the constant lowest-order volume form, which is dropped (the
  printed form is garbled; a constant factor per tet does not change the
  constraint).  These span the polynomials of degree p-1 on each tet, where
  div W2 lives, so [div] b = 0 holds exactly iff div b = 0.
* [*3] is invertible, so the constraint is imposed as [~div] b = 0.
* mu^-1 multiplies both sides of the Galerkin system, so it is left out.

Test infrastructure only: part of the CPU oracle, which the product library
never imports.
"""

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import basis, basis3
from .quadrature import tet_rule


def w3_spec(order):
    """Multi-indices (a, b, c, d), all >= 1, summing to order + 3."""
    n = order + 3
    out = []
    for a in range(1, n):
        for b in range(1, n - a):
            for c in range(1, n - a - b):
                d = n - a - b - c
                if d >= 1:
                    out.append((a, b, c, d))
    return out


def w3(order, lam):
    """[..., n3] values of the order-p volume functions (constant form dropped)."""
    vals = []
    for idx in w3_spec(order):
        m = np.ones(lam.shape[:-1])
        for v, i in enumerate(idx):
            pv, _ = basis3.silvester_hat(i, order + 3, lam[..., v])
            m = m * pv
        vals.append(m)
    return np.stack(vals, axis=-1)


def matrices(topo, g, vol):
    """[*3] (block diagonal), [~div] (N3 x N2) and the W2 mass <W2, W2>."""
    lam_q, w_q = tet_rule(topo.order + 3)
    n3 = len(w3_spec(topo.order))
    nt = topo.n_tets
    W3 = w3(topo.order, lam_q)                                # [Q, n3]
    rows, cols, v_s3, r_d, c_d, v_d = [], [], [], [], [], []
    for t in range(nt):
        gg = np.broadcast_to(g[t], (len(lam_q), 4, 3))
        dv = basis.div_w2(topo.order, lam_q, gg)              # [Q, n2]
        sc = 6.0 * vol[t]
        s3 = sc * np.einsum("q,qi,qj->ij", w_q, W3, W3)
        dd = sc * np.einsum("q,qi,qj->ij", w_q, W3, dv)
        base = t * n3
        for i in range(n3):
            for j in range(n3):
                rows.append(base + i); cols.append(base + j); v_s3.append(s3[i, j])
            for j in range(dd.shape[1]):
                if dd[i, j] != 0.0:
                    r_d.append(base + i); c_d.append(topo.dof2[t, j]); v_d.append(dd[i, j])
    S3 = sp.csr_matrix((v_s3, (rows, cols)), shape=(nt * n3, nt * n3))
    Dv = sp.csr_matrix((v_d, (r_d, c_d)), shape=(nt * n3, topo.n2))
    from .assemble import mass2, MU0
    M2 = mass2(topo, g, vol) * MU0                            # <W2_i, W2_j>
    return S3, Dv, M2


def load(topo, g, vol, field):
    """f_i = <W2_i, B> by the tet rule of p + 3 points per direction."""
    lam_q, w_q = tet_rule(topo.order + 3)
    f = np.zeros(topo.n2)
    x_all = np.einsum("qk,tkd->tqd", lam_q, topo.xyz[topo.tets])
    for t in range(topo.n_tets):
        gg = np.broadcast_to(g[t], (len(lam_q), 4, 3))
        w = basis.w2(topo.order, lam_q, gg)
        np.add.at(f, topo.dof2[t], 6.0 * vol[t] * np.einsum("q,qik,qk->i", w_q, w, field(x_all[t])))
    return f


def project(topo, g, vol, field, constrained=True):
    """W2 coefficients of the impressed field: Galerkin, or constrained by
    Gauss's magnetic law (eq. conB)."""
    S3, Dv, M2 = matrices(topo, g, vol)
    f = load(topo, g, vol, field)
    if not constrained:
        return spla.spsolve(M2.tocsc(), f)
    n2, n3 = topo.n2, Dv.shape[0]
    # div maps W2 (no boundary condition) onto the discontinuous degree-(p-1)
    # polynomials, so [~div] has full row rank and the saddle-point matrix is
    # invertible
    K = sp.bmat([[M2, Dv.T], [Dv, None]]).tocsc()
    rhs = np.concatenate([f, np.zeros(n3)])
    return spla.spsolve(K, rhs)[:n2]


def errors(topo, g, c, vol, bcoef, field):
    """Relative L2 error of the reconstruction and the L2 norm of its
    divergence (relative to the field's L2 norm per unit length)."""
    lam_q, w_q = tet_rule(topo.order + 3)
    x_all = np.einsum("qk,tkd->tqd", lam_q, topo.xyz[topo.tets])
    num = den = div2 = 0.0
    for t in range(topo.n_tets):
        gg = np.broadcast_to(g[t], (len(lam_q), 4, 3))
        Bh = np.einsum("i,qik->qk", bcoef[topo.dof2[t]], basis.w2(topo.order, lam_q, gg))
        F = field(x_all[t])
        sc = 6.0 * vol[t]
        num += sc * np.sum(w_q * np.sum((Bh - F) ** 2, axis=1))
        den += sc * np.sum(w_q * np.sum(F ** 2, axis=1))
        dv = basis.div_w2(topo.order, lam_q, gg) @ bcoef[topo.dof2[t]]
        div2 += sc * np.sum(w_q * dv ** 2)
    return float(np.sqrt(num / den)), float(np.sqrt(div2 / den))

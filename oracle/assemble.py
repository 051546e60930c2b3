"""Global matrices of the discrete de Rham complex (Section III-A).

* Hodge matrices [*eps]_ij = <W1_i, eps0 W1_j> and [*mu^-1]_ij =
  <W2_i, mu0^-1 W2_j> (Section III-A, the Hodge matrix definitions);
* the curl-curl matrix K_ij = <curl W1_i, mu0^-1 curl W1_j>, which equals
  C^T [*mu^-1] C because curl W1 lies in span W2;
* the exact-sequence maps: grad W0_k = sum_i D_ik W1_i and
  curl W1_j = sum_f C_fj W2_f.  The paper notes that beyond the lowest order
  these "cannot be written by inspection"; here they are found on the
  reference tet by least squares (the bases are written in barycentric
  coordinates and their gradients, so the coefficients are the same on every
  tet) and assembled, with a check that shared entities get equal values;
* the nodal Laplacian L = D^T [*eps] D and the nodal load <W0_k, 1>;
* the surface impedance matrix of Section III-A,
  [*_I]_ij = <n x W1_i, Y n x W1_j> over the impedance faces (eq.
  impedanceBC).  Reading: the printed weight is mu^-1, but only the
  admittance Y makes the term commensurate with [*eps] d/dt e (the weak form
  of Ampere's law picks up  Y int (n x W_i).(n x E) dS  from n x H =
  Y n x n x E); Y = Y0 = sqrt(eps0 / mu0), free space, for the first-order
  absorbing condition.

Integrals use the collapsed-cube rule with p + 2 points per direction (exact
for degree 2p + 1 >= 2p).

Test infrastructure only: part of the CPU oracle, which the product library
never imports.
"""

import numpy as np
import scipy.sparse as sp

from . import basis
from .quadrature import tet_rule, tri_rule

EPS0 = 8.8541878128e-12
MU0 = 1.25663706212e-6
Y0 = (EPS0 / MU0) ** 0.5

G_REF = np.array([[-1.0, -1.0, -1.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])


def _ref_samples(n=4):
    lam, _ = tet_rule(n)
    g = np.broadcast_to(G_REF, (len(lam), 4, 3))
    return lam, g


def _lstsq_map(target, base):
    """Coefficients X with target[:, k] = base @ X[:, k]; target/base are
    stacked [points*3, n].  Returns X and the max residual."""
    x, *_ = np.linalg.lstsq(base, target, rcond=None)
    res = np.max(np.abs(base @ x - target)) if target.size else 0.0
    x[np.abs(x) < 1e-13] = 0.0
    return x, res


def local_grad_map(order):
    """D_loc [n1, n0]: grad W0_k = sum_i D_loc[i, k] W1_i."""
    lam, g = _ref_samples()
    w1 = basis.w1(order, lam, g)            # [Q, n1, 3]
    gw0 = basis.grad_w0(order, lam, g)      # [Q, n0, 3]
    base = np.transpose(w1, (0, 2, 1)).reshape(-1, w1.shape[1])
    tgt = np.transpose(gw0, (0, 2, 1)).reshape(-1, gw0.shape[1])
    return _lstsq_map(tgt, base)


def local_curl_map(order):
    """C_loc [n2, n1]: curl W1_j = sum_f C_loc[f, j] W2_f."""
    lam, g = _ref_samples()
    w2 = basis.w2(order, lam, g)
    cw1 = basis.curl_w1(order, lam, g)
    base = np.transpose(w2, (0, 2, 1)).reshape(-1, w2.shape[1])
    tgt = np.transpose(cw1, (0, 2, 1)).reshape(-1, cw1.shape[1])
    return _lstsq_map(tgt, base)


def _assemble_map(rows_dof, cols_dof, loc, n_rows, n_cols):
    """Global matrix with G[rows_dof[t,i], cols_dof[t,k]] = loc[i,k] for every
    tet t; raises if two tets disagree on a shared entry."""
    val = {}
    for t in range(len(rows_dof)):
        for i in range(loc.shape[0]):
            for k in range(loc.shape[1]):
                x = loc[i, k]
                if x == 0.0:
                    continue
                key = (int(rows_dof[t, i]), int(cols_dof[t, k]))
                old = val.get(key)
                if old is None:
                    val[key] = x
                elif abs(old - x) > 1e-12 * max(1.0, abs(x)):
                    raise AssertionError(f"inconsistent shared entry {key}: {old} vs {x}")
    if not val:
        return sp.csr_matrix((n_rows, n_cols))
    keys = np.array(list(val.keys()))
    return sp.csr_matrix((np.array(list(val.values())), (keys[:, 0], keys[:, 1])),
                         shape=(n_rows, n_cols))


def grad_matrix(topo):
    dloc, _ = local_grad_map(topo.order)
    return _assemble_map(topo.dof1, topo.dof0, dloc, topo.n1, topo.n0)


def curl_matrix(topo):
    cloc, _ = local_curl_map(topo.order)
    return _assemble_map(topo.dof2, topo.dof1, cloc, topo.n2, topo.n1)


def _element_integrals(topo, g, vol, kind, chunk=2048):
    """Per-tet integrals of products of basis values; kind in
    {'m1','k','m2','w0'}."""
    lam_q, w_q = tet_rule(topo.order + 2)   # exact for degree 2p + 1
    out = []
    for s in range(0, topo.n_tets, chunk):
        gg = g[s:s + chunk][:, None, :, :]
        lq = lam_q[None, :, :]
        scale = 6.0 * vol[s:s + chunk]
        if kind == "m1":
            f = basis.w1(topo.order, lq, gg)
        elif kind == "k":
            f = basis.curl_w1(topo.order, lq, gg)
        elif kind == "m2":
            f = basis.w2(topo.order, lq, gg)
        else:
            f = basis.w0(topo.order, np.broadcast_to(lq, (len(gg),) + lam_q.shape))
            out.append(np.einsum("q,tqi->ti", w_q, f) * scale[:, None])
            continue
        out.append(np.einsum("q,tqik,tqjk->tij", w_q, f, f) * scale[:, None, None])
    return np.concatenate(out, axis=0)


def _assemble_sum(dofs, ke, n):
    r = np.repeat(dofs[:, :, None], dofs.shape[1], axis=2).ravel()
    c = np.repeat(dofs[:, None, :], dofs.shape[1], axis=1).ravel()
    return sp.csr_matrix((ke.ravel(), (r, c)), shape=(n, n))


def mass1(topo, g, vol):
    """[*eps] (Section III-A)."""
    return _assemble_sum(topo.dof1, EPS0 * _element_integrals(topo, g, vol, "m1"), topo.n1)


def curlcurl(topo, g, vol):
    """K = <curl W1, mu0^-1 curl W1>."""
    return _assemble_sum(topo.dof1, _element_integrals(topo, g, vol, "k") / MU0, topo.n1)


def mass2(topo, g, vol):
    """[*mu^-1] (Section III-A)."""
    return _assemble_sum(topo.dof2, _element_integrals(topo, g, vol, "m2") / MU0, topo.n2)


def nodal_load(topo, g, vol):
    """<W0_k, 1>."""
    loc = _element_integrals(topo, g, vol, "w0")
    out = np.zeros(topo.n0)
    np.add.at(out, topo.dof0.ravel(), loc.ravel())
    return out


def impedance(topo, g, Y=None):
    """[*_I]_ij = Y <n x W1_i, n x W1_j> over the faces tagged impedance: on
    each such face (the face opposite local vertex i of its tet, where
    lambda_i = 0) the tangential part W - (W.n) n of every local W1 function
    is integrated against every other with the collapsed triangle rule of
    order + 2 points per direction (exact for degree 2p + 2)."""
    Y = Y0 if Y is None else Y
    n1 = topo.n1
    rows, cols, vals = [], [], []
    lam2, w2 = tri_rule(topo.order + 2)
    for f in np.nonzero(topo.imp_face)[0]:
        tt, i = None, None
        hit = np.nonzero(topo.tet_faces == f)
        tt, i = int(hit[0][0]), int(hit[1][0])
        verts = [k for k in range(4) if k != i]
        lam = np.zeros((len(w2), 4))
        for j, k in enumerate(verts):
            lam[:, k] = lam2[:, j]
        P = topo.xyz[topo.tets[tt]]
        area = 0.5 * np.linalg.norm(np.cross(P[verts[1]] - P[verts[0]], P[verts[2]] - P[verts[0]]))
        nrm = g[tt, i] / np.linalg.norm(g[tt, i])
        W = basis.w1(topo.order, lam, np.broadcast_to(g[tt], (len(w2), 4, 3)))
        Wt = W - np.einsum("qjk,k->qj", W, nrm)[:, :, None] * nrm[None, None, :]
        ke = Y * 2.0 * area * np.einsum("q,qak,qbk->ab", w2, Wt, Wt)
        d = topo.dof1[tt]
        rows.append(np.repeat(d, len(d)))
        cols.append(np.tile(d, len(d)))
        vals.append(ke.ravel())
    if not rows:
        return sp.csr_matrix((n1, n1))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n1, n1))

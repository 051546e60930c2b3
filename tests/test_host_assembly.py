"""The library's host set-up (setup.cpp) against the oracle, on the CPU: a small
harness (host_dump.cpp) built with the library's host source writes the
assembled operators of a jittered box with one impedance wall, at orders 1-3.

Tolerances: rel 1e-13 (exact rational element tables on the host, a
Gauss-Legendre rule exact for the integrands in the oracle; only rounding
differs).  Checked: [*eps], the curl-curl matrix, the curl and gradient maps,
[*mu^-1], the impedance matrix, the preconditioner's gradient space with the
impedance wall's W0 DOFs and its Laplacian (mass and impedance parts), the
projection's [~div], the PEC and boundary masks, the load's quadrature rule,
and the injection table (bit-exact: the re-injection's sampling reads it).
"""

import os
import subprocess

import numpy as np
import pytest
import scipy.sparse as sp

import workloads
from oracle import assemble, basis, geometry, project, topology

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    d = tmp_path_factory.mktemp("host")
    exe = d / "host_dump"
    subprocess.run(["g++", "-O1", "-std=c++17", "-ffp-contract=off", "-pthread",
                    "-I", os.path.join(ROOT, "include"), os.path.join(HERE, "host_dump.cpp"),
                    os.path.join(ROOT, "paper_2111_12411_gb300", "csrc", "setup.cpp"), "-o", str(exe)],
                   check=True, capture_output=True)
    return exe


def _read(f):
    nr, nc = np.fromfile(f, np.int32, 2)
    nnz = int(np.fromfile(f, np.int64, 1)[0])
    rp = np.fromfile(f, np.int32, nr + 1)
    ci = np.fromfile(f, np.int32, nnz)
    v = np.fromfile(f, np.float64, nnz)
    return sp.csr_matrix((v, ci, rp), shape=(nr, nc))


def _rel(a, b):
    a, b = np.asarray(a.todense() if sp.issparse(a) else a), np.asarray(b.todense() if sp.issparse(b) else b)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _mesh():
    xyz, tets = workloads.kuhn_box(3, 3, 3, jitter=0.1, seed=21)
    tag = np.zeros((len(tets), 4), dtype=np.int32)
    for i in range(4):
        X = xyz[np.delete(tets, i, axis=1)][:, :, 0]
        tag[np.all(np.abs(X - 1.0) < 1e-12, axis=1), i] = 1  # impedance wall x = 1
        tag[np.all(np.abs(X) < 1e-12, axis=1), i] = 4        # injection faces on x = 0
    return xyz, tets, tag


def _w0_on_pec_faces(t, order, g):
    """W0 DOFs whose function is nonzero somewhere on a PEC face (sampled on
    the face) - the DOFs the preconditioner's gradient space must leave out."""
    on = np.zeros(t.n0, dtype=bool)
    pec_face = t.boundary_face & ~t.imp_face
    rng = np.random.default_rng(0)
    for tt in range(t.n_tets):
        for k in range(4):
            if not pec_face[t.tet_faces[tt, k]]:
                continue
            lam = rng.dirichlet(np.ones(3), size=5)
            L = np.insert(lam, k, 0.0, axis=1)  # points on the face opposite local vertex k
            w = basis.w0(order, L)
            on[t.dof0[tt][np.any(np.abs(w) > 1e-12, axis=0)]] = True
    return on


@pytest.mark.parametrize("order", [1, 2, 3])
def test_host_operators_match_oracle(harness, tmp_path, order):
    xyz, tets, tag = _mesh()
    mesh = tmp_path / "mesh.bin"
    with open(mesh, "wb") as f:
        np.array([len(xyz), len(tets)], np.int32).tofile(f)
        np.ascontiguousarray(xyz).tofile(f)
        np.ascontiguousarray(tets, np.int32).tofile(f)
        tag.tofile(f)
    out = tmp_path / "ops.bin"
    subprocess.run([str(harness), str(mesh), str(out), str(order)], check=True)
    t = topology.Topology(xyz, tets, order, tag)
    g, c, vol = geometry.barycentric_maps(t.xyz, t.tets)
    with open(out, "rb") as f:
        M, K, C, D, M2, I, DA, LA, LI, Dv = (_read(f) for _ in range(10))
        pec1 = np.fromfile(f, np.uint8, t.n1).astype(bool)
        bnd0 = np.fromfile(f, np.uint8, t.n0).astype(bool)
        nq = int(np.fromfile(f, np.int32, 1)[0])
        qlam = np.fromfile(f, np.float64, 4 * nq).reshape(nq, 4)
        qw = np.fromfile(f, np.float64, nq)
        nf = int(np.fromfile(f, np.int32, 1)[0])
        ixyz = np.fromfile(f, np.float64, 9 * nf).reshape(nf, 3, 3)
        itet = np.fromfile(f, np.int32, nf)
        icum = np.fromfile(f, np.float64, nf)
    assert np.array_equal(pec1, t.pec1) and np.array_equal(bnd0, t.bnd0)
    fr, ii = t.free1, t.interior0
    Mo = assemble.mass1(t, g, vol)[fr][:, fr]
    Io = assemble.impedance(t, g)[fr][:, fr]
    assert _rel(M[fr][:, fr], Mo) < 1e-13
    assert _rel(K[fr][:, fr], assemble.curlcurl(t, g, vol)[fr][:, fr]) < 1e-13
    assert _rel(C[:, fr], assemble.curl_matrix(t)[:, fr]) < 1e-13
    Do = assemble.grad_matrix(t)
    assert _rel(D[:, ii], Do[:, ii]) < 1e-13
    assert _rel(M2, assemble.mass2(t, g, vol)) < 1e-13
    assert _rel(I[fr][:, fr], Io) < 1e-13
    # the gradient space of the preconditioner: every W0 DOF off the PEC faces
    aux = ~_w0_on_pec_faces(t, order, g)
    assert aux.sum() > ii.sum()  # the impedance wall's inner W0 DOFs join the interior ones
    Da = Do[fr][:, aux]
    assert _rel(DA[fr][:, aux], Da) < 1e-13
    assert abs(DA[:, ~aux]).sum() == 0 and abs(DA[~fr]).sum() == 0
    assert _rel(LA[aux][:, aux], (Da.T @ Mo @ Da)) < 1e-13
    assert _rel(LI[aux][:, aux], (Da.T @ Io @ Da)) < 1e-13
    # the projection's divergence operator against the W3 volume functions
    S3, Dvo, M2o = project.matrices(t, g, vol)
    assert _rel(Dv, Dvo) < 1e-13
    # the load's conical Gauss rule (nodes from Newton on P_n against numpy's
    # Legendre-Gauss rule) and the injection table, bit-exact where the
    # re-injection's sampling reads it
    from oracle import inject, quadrature
    ql, qwo = quadrature.tet_rule(order + 3)
    assert np.abs(qlam - ql).max() < 1e-15 and np.abs(qw - qwo).max() < 1e-16
    verts, owner, cum = inject.face_table(t)
    assert nf == len(owner) == 18
    assert np.array_equal(ixyz, verts) and np.array_equal(itet, owner) and np.array_equal(icum, cum)

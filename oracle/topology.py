"""Mesh complex K = {N, E, F, T} and degree-of-freedom numbering.

Follows Section III-A ("Discretization in Space"): the domain is a collection
of tetrahedra with N_n nodes, N_e edges, N_f faces and N_t tets; each tet
carries W0/W1/W2 basis functions of order k (DOF counts in Section III-A and
the Appendix).

Canonical numbering (a reading: the paper states none):

* every tet's four vertices are sorted by global node id; local vertex i is the
  i-th smallest.  Edges and faces are oriented from the smaller to the larger
  global id, so local and global orientations agree and all signs are +1;
* edges are the unique sorted pairs, faces the unique sorted triples, both in
  lexicographic order;
* local edge j is ``LOCAL_EDGES[j]``; local face i is the face opposite local
  vertex i (``LOCAL_FACES[i]``);
* order 1: W1 DOF = edge id, W2 DOF = face id, W0 DOF = node id;
* order 2: W1 DOFs are ``2*edge + v`` (v=0: multiplier attached to the lower
  vertex, v=1: to the upper) then ``2*N_e + 2*face + v``; W2 DOFs are
  ``3*face + v`` then ``3*N_f + 3*tet + i``; W0 DOFs are nodes then
  ``N_n + edge`` (mid-edge Lagrange nodes).

Boundary conditions (Section II, eq. bceq): every boundary face is either
perfect electric conductor (Dirichlet n x E = 0, tag 0, the default) or
impedance (eq. impedanceBC with Psi_I = 0, the first-order absorbing
condition, tag 1).  ``bface_tag[t, i]`` tags the face opposite the i-th vertex
of tet t as given (before sorting); it is read for boundary faces only.  A W1
DOF is held at 0 when its edge or face lies on a PEC face (an edge shared by
a PEC and an impedance face is PEC); DOFs on impedance faces only are free.
W0 boundary DOFs (Dirichlet for the nodal Laplacian and the Gauss residual)
remain all boundary nodes.

Particle walls (the paper is silent on what happens to particles at walls):
a boundary face reflects particles specularly unless its tag has bit 2 set
(absorbing: the path ends on the face and the particle is re-injected).  Bit 4
marks an injection face (particles are re-injected on such faces; an
injection face reflects unless it is also absorbing).  Bit 1 is the field
condition above, so a tag is (impedance) | 2 (absorb) | 4 (inject).

Test infrastructure only: part of the CPU oracle, which the product library
never imports.
"""

import numpy as np

LOCAL_EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))
LOCAL_FACES = ((1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2))


class MeshError(ValueError):
    pass


class Topology:
    """Entities, adjacency and DOF maps of a tet mesh for a given order."""

    def __init__(self, xyz, tets, order, bface_tag=None):
        if order not in (1, 2, 3):
            raise ValueError("order must be 1, 2 or 3")
        xyz = np.asarray(xyz, dtype=np.float64)
        t_in = np.asarray(tets, dtype=np.int64)
        t = np.sort(t_in, axis=1)
        if t.size and (t.min() < 0 or t.max() >= len(xyz)):
            raise MeshError("tet references a node out of range")
        if np.any(t[:, 1:] == t[:, :-1]):
            raise MeshError("tet with a repeated vertex")
        self.order = order
        self.xyz = xyz
        self.tets = t
        nt = len(t)
        self.n_nodes, self.n_tets = len(xyz), nt

        e_all = t[:, LOCAL_EDGES].reshape(-1, 2)
        self.edges, inv = np.unique(e_all, axis=0, return_inverse=True)
        self.tet_edges = inv.reshape(nt, 6)
        f_all = t[:, LOCAL_FACES].reshape(-1, 3)
        self.faces, inv = np.unique(f_all, axis=0, return_inverse=True)
        self.tet_faces = inv.reshape(nt, 4)
        self.n_edges, self.n_faces = len(self.edges), len(self.faces)

        # face -> the (at most two) tets that own it
        owners = np.full((self.n_faces, 2), -1, dtype=np.int64)
        owner_face = np.full((self.n_faces, 2), -1, dtype=np.int64)
        count = np.zeros(self.n_faces, dtype=np.int64)
        for tt in range(nt):
            for i in range(4):
                f = self.tet_faces[tt, i]
                if count[f] >= 2:
                    raise MeshError("face shared by more than two tets")
                owners[f, count[f]] = tt
                owner_face[f, count[f]] = i
                count[f] += 1
        self.tet2tet = np.full((nt, 4), -1, dtype=np.int64)
        self.tet2face = np.full((nt, 4), -1, dtype=np.int64)  # local face index in the neighbour
        for f in np.nonzero(count == 2)[0]:
            a, b = owners[f]
            ia, ib = owner_face[f]
            self.tet2tet[a, ia], self.tet2face[a, ia] = b, ib
            self.tet2tet[b, ib], self.tet2face[b, ib] = a, ia
        self.boundary_face = count == 1
        # boundary face tags: -1 interior, 0 PEC, 1 impedance; particle walls
        self.face_tag = np.where(self.boundary_face, 0, -1).astype(np.int64)
        self.absorb_face = np.zeros(self.n_faces, dtype=bool)
        self.inject_face = np.zeros(self.n_faces, dtype=bool)
        if bface_tag is not None:
            tag_in = np.asarray(bface_tag, dtype=np.int64).reshape(nt, 4)
            if np.any((tag_in < 0) | (tag_in > 7)):
                raise ValueError("face tags are 0..7: 1 impedance | 2 absorb | 4 inject")
            for tt in range(nt):
                for i in range(4):
                    tri = np.sort(np.delete(t_in[tt], i))
                    # the face of the sorted tet that has the same three vertices
                    j = int(np.nonzero(t[tt] == t_in[tt, i])[0][0])
                    f = self.tet_faces[tt, j]
                    assert np.array_equal(self.faces[f], tri)
                    if self.boundary_face[f]:
                        self.face_tag[f] = tag_in[tt, i] & 1
                        self.absorb_face[f] = bool(tag_in[tt, i] & 2)
                        self.inject_face[f] = bool(tag_in[tt, i] & 4)
        self.imp_face = self.face_tag == 1
        # absorbing wall per (tet, local face) for the walk
        self.tet_absorb = self.absorb_face[self.tet_faces] & self.boundary_face[self.tet_faces]
        pf = self.faces[self.face_tag == 0]
        pedge = set()
        for (a, b, c) in pf:
            pedge.update([(a, b), (a, c), (b, c)])
        self.pec_edge = np.zeros(len(self.edges), dtype=bool)
        if pedge:
            pe = np.array(sorted(pedge), dtype=np.int64)
            key = self.edges[:, 0] * self.n_nodes + self.edges[:, 1]
            self.pec_edge = np.isin(key, pe[:, 0] * self.n_nodes + pe[:, 1])
        bf = self.faces[self.boundary_face]
        self.boundary_node = np.zeros(self.n_nodes, dtype=bool)
        self.boundary_node[bf.ravel()] = True
        bedge = set()
        for (a, b, c) in bf:
            bedge.update([(a, b), (a, c), (b, c)])
        self.boundary_edge = np.zeros(self.n_edges, dtype=bool)
        if bedge:
            be = np.array(sorted(bedge), dtype=np.int64)
            key = self.edges[:, 0] * self.n_nodes + self.edges[:, 1]
            bkey = be[:, 0] * self.n_nodes + be[:, 1]
            self.boundary_edge = np.isin(key, bkey)
        self._dofs()

    def _dofs(self):
        ne, nf, nt, nn = self.n_edges, self.n_faces, self.n_tets, self.n_nodes
        te, tf = self.tet_edges, self.tet_faces
        if self.order == 1:
            self.n1, self.n2, self.n0 = ne, nf, nn
            self.dof1 = te.copy()
            self.dof2 = tf.copy()
            self.dof0 = self.tets.copy()
            self.pec1 = self.pec_edge.copy()
            self.bnd0 = self.boundary_node.copy()
        elif self.order == 3:
            # basis3: W1 3 per edge, 6 per face, 3 per tet; W2 6 per face,
            # 12 per tet; W0 nodes, 2 per edge, 1 per face
            self.n1 = 3 * ne + 6 * nf + 3 * nt
            self.n2 = 6 * nf + 12 * nt
            self.n0 = nn + 2 * ne + nf
            d1 = np.zeros((nt, 45), dtype=np.int64)
            for j in range(6):
                for v in range(3):
                    d1[:, 3 * j + v] = 3 * te[:, j] + v
            for i in range(4):
                for v in range(6):
                    d1[:, 18 + 6 * i + v] = 3 * ne + 6 * tf[:, i] + v
            for v in range(3):
                d1[:, 42 + v] = 3 * ne + 6 * nf + 3 * np.arange(nt) + v
            self.dof1 = d1
            d2 = np.zeros((nt, 36), dtype=np.int64)
            for i in range(4):
                for v in range(6):
                    d2[:, 6 * i + v] = 6 * tf[:, i] + v
            for v in range(12):
                d2[:, 24 + v] = 6 * nf + 12 * np.arange(nt) + v
            self.dof2 = d2
            d0 = np.zeros((nt, 20), dtype=np.int64)
            d0[:, :4] = self.tets
            for j in range(6):
                for v in range(2):
                    d0[:, 4 + 2 * j + v] = nn + 2 * te[:, j] + v
            for i in range(4):
                d0[:, 16 + i] = nn + 2 * ne + tf[:, i]
            self.dof0 = d0
            pec = np.zeros(self.n1, dtype=bool)
            for v in range(3):
                pec[3 * np.nonzero(self.pec_edge)[0] + v] = True
            pf = np.nonzero(self.face_tag == 0)[0]
            for v in range(6):
                pec[3 * ne + 6 * pf + v] = True
            self.pec1 = pec
            bf = np.nonzero(self.boundary_face)[0]
            bnd_face = np.zeros(nf, dtype=bool)
            bnd_face[bf] = True
            self.bnd0 = np.concatenate([self.boundary_node, np.repeat(self.boundary_edge, 2), bnd_face])
        else:
            self.n1 = 2 * ne + 2 * nf
            self.n2 = 3 * nf + 3 * nt
            self.n0 = nn + ne
            d1 = np.zeros((nt, 20), dtype=np.int64)
            d1[:, 0:12:2] = 2 * te
            d1[:, 1:12:2] = 2 * te + 1
            d1[:, 12:20:2] = 2 * ne + 2 * tf
            d1[:, 13:20:2] = 2 * ne + 2 * tf + 1
            self.dof1 = d1
            d2 = np.zeros((nt, 15), dtype=np.int64)
            for v in range(3):
                d2[:, v:12:3] = 3 * tf + v
            for i in range(3):
                d2[:, 12 + i] = 3 * nf + 3 * np.arange(nt) + i
            self.dof2 = d2
            self.dof0 = np.concatenate([self.tets, nn + te], axis=1)
            pec = np.zeros(self.n1, dtype=bool)
            be = np.nonzero(self.pec_edge)[0]
            pec[2 * be] = True
            pec[2 * be + 1] = True
            bfid = np.nonzero(self.face_tag == 0)[0]
            pec[2 * ne + 2 * bfid] = True
            pec[2 * ne + 2 * bfid + 1] = True
            self.pec1 = pec
            self.bnd0 = np.concatenate([self.boundary_node, self.boundary_edge])
        self.free1 = ~self.pec1
        self.interior0 = ~self.bnd0

"""Structured tetrahedral meshes used as synthetic workloads.

* ``kuhn_box``: an nx x ny x nz box of hexahedra, each cut into the 6 Kuhn
  (path) simplices, which makes the triangulation conforming across all cells;
  interior nodes may be jittered (seeded).
* ``polar_tube``: a cylinder meshed on a polar grid.  Rings 1..n_rad-1 are
  hexahedra cut by the Kuhn rule in (radial, azimuthal, axial) index space
  (conforming across the azimuthal seam because the rule is translation
  invariant); the ring touching the axis is made of triangular prisms, each cut
  into 3 tets whose diagonals match the Kuhn cut of the neighbouring hexahedra.

Both return ``xyz`` (float64, [n_nodes, 3]) and ``tets`` (int32, [n_tets, 4]).
"""

import itertools

import numpy as np

# The 6 Kuhn simplices of the unit cube: one per permutation of the axes; each
# walks (0,0,0) -> +e_a -> +e_a+e_b -> (1,1,1).
_KUHN = []
for _perm in itertools.permutations(range(3)):
    _c = [0, 0, 0]
    _chain = [tuple(_c)]
    for _ax in _perm:
        _c[_ax] = 1
        _chain.append(tuple(_c))
    _KUHN.append(_chain)


def tet_volumes(xyz, tets):
    """Signed volumes of the tets (float64)."""
    p = xyz[tets]
    a = p[:, 1] - p[:, 0]
    b = p[:, 2] - p[:, 0]
    c = p[:, 3] - p[:, 0]
    return np.einsum("ij,ij->i", a, np.cross(b, c)) / 6.0


def _kuhn_cells(nx, ny, nz, node_id, wrap_y=False):
    tets = []
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                for chain in _KUHN:
                    tet = []
                    for (di, dj, dk) in chain:
                        jj = j + dj
                        if wrap_y:
                            jj %= ny
                        tet.append(node_id(i + di, jj, k + dk))
                    tets.append(tet)
    return tets


def kuhn_box(nx, ny, nz, lengths=(1.0, 1.0, 1.0), jitter=0.0, seed=0,
             min_vol_frac=0.05, max_tries=200):
    """Kuhn-split box mesh ``[0,Lx]x[0,Ly]x[0,Lz]``.

    ``jitter`` is the half-width of the uniform displacement of each interior
    node, as a fraction of the cell spacing along each axis.  A displaced node
    is drawn again while any tet touching it would have a volume below
    ``min_vol_frac`` times the nominal volume ``hx*hy*hz/6``.
    """
    lx, ly, lz = lengths
    hx, hy, hz = lx / nx, ly / ny, lz / nz
    ii, jj, kk = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1),
                             np.arange(nz + 1), indexing="ij")
    # node id = i + (nx+1)*(j + (ny+1)*k)
    n_nodes = (nx + 1) * (ny + 1) * (nz + 1)
    xyz = np.zeros((n_nodes, 3))
    ids = ii + (nx + 1) * (jj + (ny + 1) * kk)
    xyz[ids.ravel(), 0] = ii.ravel() * hx
    xyz[ids.ravel(), 1] = jj.ravel() * hy
    xyz[ids.ravel(), 2] = kk.ravel() * hz

    def nid(i, j, k):
        return i + (nx + 1) * (j + (ny + 1) * k)

    tets = np.asarray(_kuhn_cells(nx, ny, nz, nid), dtype=np.int64)
    vol = tet_volumes(xyz, tets)
    orient = np.sign(vol)

    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        nominal = hx * hy * hz / 6.0
        incident = [[] for _ in range(n_nodes)]
        for t, tet in enumerate(tets):
            for v in tet:
                incident[v].append(t)
        amp = np.array([hx, hy, hz]) * jitter
        for k in range(1, nz):
            for j in range(1, ny):
                for i in range(1, nx):
                    v = nid(i, j, k)
                    base = xyz[v].copy()
                    inc = np.asarray(incident[v])
                    for _ in range(max_tries):
                        xyz[v] = base + rng.uniform(-1.0, 1.0, 3) * amp
                        sv = tet_volumes(xyz, tets[inc]) * orient[inc]
                        if np.all(sv > min_vol_frac * nominal):
                            break
                    else:
                        xyz[v] = base
    return xyz, tets.astype(np.int32)


def polar_tube(n_az=24, n_rad=12, n_ax=80, radius=0.01, length=0.10):
    """Cylinder of ``radius`` x ``length`` along +z on a polar grid."""
    n_axis = n_ax + 1

    def ring(i, j, k):  # i in 1..n_rad, j mod n_az, k in 0..n_ax
        return n_axis + (k * n_az + (j % n_az)) * n_rad + (i - 1)

    def axis(k):
        return k

    n_nodes = n_axis + n_rad * n_az * (n_ax + 1)
    xyz = np.zeros((n_nodes, 3))
    z = np.arange(n_ax + 1) * (length / n_ax)
    xyz[:n_axis, 2] = z
    for k in range(n_ax + 1):
        for j in range(n_az):
            th = 2.0 * np.pi * j / n_az
            for i in range(1, n_rad + 1):
                r = radius * i / n_rad
                xyz[ring(i, j, k)] = (r * np.cos(th), r * np.sin(th), z[k])

    tets = []
    for k in range(n_ax):
        for j in range(n_az):
            A, A1 = axis(k), axis(k + 1)
            P, Q = ring(1, j, k), ring(1, j + 1, k)
            P1, Q1 = ring(1, j, k + 1), ring(1, j + 1, k + 1)
            tets += [[A, P, Q, Q1], [A, P, Q1, P1], [A, P1, Q1, A1]]
    # hexahedral rings: Kuhn rule in (i-1, j, k) index space, j periodic
    def nid(i0, j, k):
        return ring(i0 + 1, j, k)

    tets += _kuhn_cells(n_rad - 1, n_az, n_ax, nid, wrap_y=True)
    return xyz, np.asarray(tets, dtype=np.int32)


def tube_wall_tags(xyz, tets, length, r_inject):
    """Face tags [n_tets, 4] (face opposite the i-th vertex as given) for a
    beam through a tube along +z: faces lying on z = length absorb particles
    (2), faces on z = 0 whose centroid is within r_inject of the axis are
    injection faces (4), every other face 0.  Geometry only."""
    tets = np.asarray(tets)
    tags = np.zeros(tets.shape, dtype=np.int32)
    z = xyz[:, 2]
    for i in range(4):
        others = np.delete(tets, i, axis=1)
        zf = z[others]
        cen = xyz[others].mean(axis=1)
        at_end = np.all(np.abs(zf - length) <= 1e-12 * max(1.0, abs(length)), axis=1)
        at_start = np.all(np.abs(zf) <= 1e-12 * max(1.0, abs(length)), axis=1)
        in_beam = np.hypot(cen[:, 0], cen[:, 1]) < r_inject
        tags[at_end, i] = 2
        tags[at_start & in_beam, i] = 4
    return tags


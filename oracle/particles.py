"""Particle half of the PIC cycle (Sections II, III-B).

* ``gather``: E(x) = sum_i e_i W1_i(x) and B(x) = B0 + sum_j b_j W2_j(x)
  (Section III-A field expansions; B0 is a uniform impressed field, added
  analytically).
* ``boris``: the Lorentz-force push (Section II, Newton's equations with
  F = q(E + v x B)), in the leapfrog rotation form of Boris (1970); positions
  move on straight chords x^{n+1} = x^n + dt v^{n+1/2}.  (The paper's own push
  is Adams-Bashforth 4 on a quartic path; the straight-chord form is the one
  this library implements.)
* ``walk_deposit``: the trajectory is split into sub-segments, one per tet
  crossed, by intersecting the chord with the faces (exit face = the face with
  lambda_i(b) < 0, entry face excluded, of smallest crossing parameter
  s_i = lambda_i(a) / (lambda_i(a) - lambda_i(b)), ties to the lowest local
  index).  On each sub-segment the current DOFs receive
  q w int W1_i(r(s)) . (b - a) ds (Section III-B: g_i = <W1_i, G>, with an
  integration rule exact for the product of the basis and the path): the
  integrand has degree p in s, so 1 Gauss-Legendre point suffices at p=1 and
  2 at p=2 and p=3.  Note grad l . (b - a) = l(b) - l(a), so no geometry is needed
  beyond lambda at the two ends.  Walls (faces without neighbour) reflect the
  particle specularly at the hit point; the path stays a connected polyline.
* ``measure_rho``: rho_k = q w sum_p W0_k(x_p) (Section III-A: charge
  measured with the nodal basis).

Every float operation is written out in a fixed order (one rounding each).

Test infrastructure only: part of the CPU oracle, which the product library
never imports.
"""

import numpy as np

from . import basis, basis3, geometry
from .topology import LOCAL_EDGES

GL2_X = 0.5773502691896257645  # 1/sqrt(3): 2-point Gauss-Legendre abscissa on [-1, 1]
FNV_OFFSET = np.uint64(14695981039346656037)
FNV_PRIME = np.uint64(1099511628211)


def gather(topo, g_all, c_all, e, b, B0, x, tet):
    g, c = g_all[tet], c_all[tet]
    lam = geometry.lam(g, c, x)
    E = basis.combine(e[topo.dof1[tet]], basis.w1(topo.order, lam, g))
    Bs = basis.combine(b[topo.dof2[tet]], basis.w2(topo.order, lam, g))
    B = Bs + np.asarray(B0, dtype=np.float64)
    return E, B


def boris(v, E, B, q, m, dt):
    h = ((q / m) * dt) * 0.5
    eh = E * h
    vm = v + eh
    t = B * h
    t2 = (t[:, 0] * t[:, 0] + t[:, 1] * t[:, 1]) + t[:, 2] * t[:, 2]
    s = t * (2.0 / (1.0 + t2))[:, None]
    vp = vm + geometry.cross(vm, t)
    vplus = vm + geometry.cross(vp, s)
    return vplus + eh


def _segment_currents(order, la, lb, s0, s1, qw):
    """q w int_{s0}^{s1} W1_j(r(s)) . (b - a) ds for every local j; [n, n1]."""
    d = lb - la
    if order == 1:
        P = la + s0[:, None] * d
        Q = la + s1[:, None] * d
        vals = [P[:, s] * Q[:, t] - P[:, t] * Q[:, s] for (s, t) in LOCAL_EDGES]
        return qw * np.stack(vals, axis=1)
    half = (s1 - s0) * 0.5
    mid = (s0 + s1) * 0.5
    r = half * GL2_X
    tot = None
    for sg in (mid - r, mid + r):
        L = la + sg[:, None] * d
        if order == 3:
            f = basis3.w1_along(L, d)
        else:
            f = []
            for (a, bb, x, kind) in basis.w1_spec(order):
                m = 3.0 * L[:, x] - 1.0 if kind == "e" else 3.0 * L[:, x]
                f.append(m * (L[:, a] * d[:, bb] - L[:, bb] * d[:, a]))
            f = np.stack(f, axis=1)
        tot = f if tot is None else tot + f
    return qw * (half[:, None] * tot)



def walk_deposit(topo, g_all, c_all, x0, x1, v, tet, qw, n1, max_cross=4096, absorb=None, dg_abs=None):
    """Walk every chord [x0, x1] through the mesh and deposit its current.

    Returns (x_end, v_end, tet_end, dg, n_cross, hash, status, absorbed)
    where ``hash`` is an FNV-1a style 64-bit hash over the 32-bit codes of
    the crossing events (new tet id, 0x80000000|face for a wall reflection,
    0xC0000000|face for an absorbing wall), ``status`` is 1 where the
    crossing cap was hit and ``absorbed`` marks paths that ended on an
    absorbing wall (``absorb`` [n_tets, 4] bool per local face of the sorted
    tet; None: every wall reflects).  An absorbed path ends at the hit point,
    its current deposited up to there.  ``dg_abs`` (optional, [n1]) receives
    the sum of the absolute values of the terms added into each DOF (the
    scale of that DOF's rounding error; the sum itself is unchanged).
    """
    n = len(x0)
    a = x0.copy()
    b = x1.copy()
    v = v.copy()
    T = np.asarray(tet, dtype=np.int64).copy()
    entry = np.full(n, -1, dtype=np.int64)
    s_in = np.zeros(n)
    ncross = np.zeros(n, dtype=np.int64)
    hsh = np.full(n, FNV_OFFSET, dtype=np.uint64)
    status = np.zeros(n, dtype=np.int32)
    absorbed = np.zeros(n, dtype=bool)
    dg = np.zeros(n1)
    act = np.arange(n)
    with np.errstate(divide="ignore", invalid="ignore"):
        while act.size:
            Ta = T[act]
            g, c = g_all[Ta], c_all[Ta]
            la = geometry.lam(g, c, a[act])
            lb = geometry.lam(g, c, b[act])
            best = np.full(act.size, -1, dtype=np.int64)
            sbest = np.full(act.size, np.inf)
            for i in range(4):
                cand = (lb[:, i] < 0.0) & (entry[act] != i)
                si = la[:, i] / (la[:, i] - lb[:, i])
                upd = cand & (si < sbest)
                sbest[upd] = si[upd]
                best[upd] = i
            done = best < 0
            s0 = s_in[act]
            s1 = np.where(done, 1.0, np.minimum(np.maximum(sbest, s0), 1.0))
            contrib = _segment_currents(topo.order, la, lb, s0, s1, qw)
            np.add.at(dg, topo.dof1[Ta].ravel(), contrib.ravel())
            if dg_abs is not None:
                np.add.at(dg_abs, topo.dof1[Ta].ravel(), np.abs(contrib).ravel())

            go = np.nonzero(~done)[0]
            if go.size:
                p = act[go]
                f = best[go]
                nb = topo.tet2tet[T[p], f]
                wall = nb < 0
                ab = wall & (absorb[T[p], f] if absorb is not None else False)
                code = np.where(ab, np.int64(0xC0000000) | f,
                                np.where(wall, np.int64(0x80000000) | f, nb)).astype(np.uint64)
                hsh[p] = (hsh[p] ^ code) * FNV_PRIME
                ncross[p] += 1
                pa_ = p[ab]
                if pa_.size:  # the path ends on the absorbing wall
                    d = b[pa_] - a[pa_]
                    b[pa_] = a[pa_] + s1[go][ab][:, None] * d
                    absorbed[pa_] = True
                inner = p[~wall]
                entry[inner] = topo.tet2face[T[inner], f[~wall]]
                T[inner] = nb[~wall]
                s_in[inner] = s1[go][~wall]
                refl = wall & ~ab
                pw = p[refl]
                if pw.size:
                    fw = f[refl]
                    gw = g_all[T[pw], fw]
                    sw = s1[go][refl]
                    d = b[pw] - a[pw]
                    hit = a[pw] + sw[:, None] * d
                    gg = geometry.dot3(gw, gw)
                    dr = d - ((2.0 * geometry.dot3(d, gw)) / gg)[:, None] * gw
                    rem = 1.0 - sw
                    b[pw] = hit + rem[:, None] * dr
                    a[pw] = hit
                    v[pw] = v[pw] - ((2.0 * geometry.dot3(v[pw], gw)) / gg)[:, None] * gw
                    s_in[pw] = 0.0
                    entry[pw] = fw
                capped = p[(ncross[p] >= max_cross) & ~absorbed[p]]
                status[capped] = 1
                keep = go[(ncross[p] < max_cross) & ~absorbed[p]]
                act = act[keep]
            else:
                act = act[:0]
    return b, v, T, dg, ncross, hsh, status, absorbed


def measure_rho(topo, g_all, c_all, x, tet, qw, rho_abs=None, rho_cnt=None):
    """rho_k = q w sum_p W0_k(x_p); rho_abs (optional, [n0]) receives the sum
    of the absolute values of the terms of each rho_k, rho_cnt (optional) the
    sum of |q w| over the particles whose tet carries DOF k."""
    g, c = g_all[tet], c_all[tet]
    lam = geometry.lam(g, c, x)
    w0 = basis.w0(topo.order, lam)
    rho = np.zeros(topo.n0)
    np.add.at(rho, topo.dof0[tet].ravel(), (qw * w0).ravel())
    if rho_abs is not None:
        np.add.at(rho_abs, topo.dof0[tet].ravel(), np.abs(qw * w0).ravel())
    if rho_cnt is not None:
        np.add.at(rho_cnt, topo.dof0[tet].ravel(), np.full(w0.size, abs(qw)))
    return rho

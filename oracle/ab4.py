"""The paper's own push: Adams-Bashforth 4 with a quartic path (Section III-B,
last paragraph: a fourth-order Adams-Bashforth push makes the particle path a
fourth-order Lagrange polynomial; the current uses an integration rule exact
for the product of the edge basis and that path).

Readings (the paper gives no further detail):

* State per particle: x^n, v^n at integer times and the history v^{n-j},
  a^{n-j} (j = 1..3); a = (q/m)(E + v x B) with E, B gathered at x^n.
  The first steps use the lower Adams-Bashforth orders (k = 1, 2, 3) while
  the history fills; all particles share the count.
* Velocity: v^{n+1} = v^n + dt sum_j beta_j a^{n-j}.
* Path: the continuous extension of the same rule for x,
  x(s) = x^n + dt int_0^s V(sigma) dsigma, s in [0, 1], where V is the
  Lagrange polynomial through (sigma = -j, v^{n-j}), j = 0..k-1: degree k in
  s, x(0) = x^n and x(1) = x^n + dt sum_j beta_j v^{n-j} = x^{n+1}.
  Coefficients x(s) = sum_m C_m s^m, C_0 = x^n, C_m = dt sum_j gam_jm v^{n-j}.
* Walk: in each tet, lambda_i(x(s)) is a polynomial in s of degree <= 4
  (lambda affine).  The particle leaves through face i at
  t_i = inf{ s in (s0, 1] : lambda_i(x(s)) < 0 }, the first parameter after
  the entry parameter s0 at which lambda_i changes sign to negative (a
  touching zero, such as a tangent path, is not a crossing).  t_i is found
  from all the polynomial's roots (companion-matrix eigenvalues,
  ``numpy.roots``): the real ones in (s0, 1) split the interval into pieces
  of constant sign, the sign of each piece is read at its middle, and the
  left end of the first negative piece is the crossing, polished by Newton
  steps on the polynomial.  Roots closer together than ROOT_MERGE (a dip
  that narrow is a graze that stays in the tet) count as one.  On the entry
  face lambda vanishes at s0 exactly, so its polynomial is divided by
  (s - s0) first and the quotient's sign decides.  The exit face is the one
  with the smallest t_i (ties to the lowest index) and the particle
  continues in the neighbour from that parameter.
* Walls: the rest of the path is mirrored in the wall plane at the hit point
  (C_0 about the hit point, C_m >= 1 as vectors), and so are v^{n+1}, v^n,
  a^n and the history, so the multistep history stays consistent with the
  reflected trajectory.
* Current: q w int_{s0}^{s1} W1_i(x(s)) . x'(s) ds with the Gauss-Legendre
  rule of 2p + 2 points (the integrand has degree p k + k - 1 <= 4p + 3);
  W1 . x' needs only lambda and lambda' = d lambda / ds along the path.
* Charge: rho^{n+1} from W0 at x^{n+1}, as for the straight chord.

Every float operation is written in a fixed order (one rounding each).

Test infrastructure only: part of the CPU oracle, which the product library
never imports.
"""

from fractions import Fraction

import numpy as np

from . import basis, geometry
from .particles import FNV_OFFSET, FNV_PRIME

ROOT_MERGE = 1e-9   # roots of one face's polynomial closer than this (in s) are one root
ROOT_IMAG = 1e-7    # a root whose imaginary part is below this (relative) is read as real
NEWTON_POLISH = 4


def _lagrange_integrals(k):
    """beta_j and gam[j][m]: int_0^s l_j(sigma) dsigma = sum_m gam[j][m] s^m,
    l_j the Lagrange basis on the nodes 0, -1, ..., -(k-1), exactly."""
    nodes = [Fraction(-j) for j in range(k)]
    gam = []
    for j in range(k):
        # polynomial coefficients of l_j(sigma) (ascending powers)
        poly = [Fraction(1)]
        den = Fraction(1)
        for i in range(k):
            if i == j:
                continue
            poly = [Fraction(0)] + poly          # sigma * poly
            for t in range(len(poly) - 1):
                poly[t] -= nodes[i] * poly[t + 1]
            den *= nodes[j] - nodes[i]
        poly = [a / den for a in poly]
        integ = [Fraction(0)] + [poly[t] / (t + 1) for t in range(len(poly))]
        gam.append(integ)
    beta = [sum(g) for g in gam]
    return beta, gam


def ab_tables(k):
    """(beta[k], gam[k][k+1]) as float64."""
    beta, gam = _lagrange_integrals(k)
    return (np.array([float(b) for b in beta]),
            np.array([[float(c) for c in row] for row in gam]))


def gauss_legendre01_n(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def _horner(coef, s):
    """coef [n, K+1, ...] ascending; s [n] -> value [n, ...]."""
    K = coef.shape[1] - 1
    p = coef[:, K]
    for m in range(K - 1, -1, -1):
        p = p * s.reshape((-1,) + (1,) * (p.ndim - 1)) + coef[:, m]
    return p


def _horner_deriv(coef, s):
    K = coef.shape[1] - 1
    if K == 0:
        return np.zeros_like(coef[:, 0])
    p = float(K) * coef[:, K]
    for m in range(K - 1, 0, -1):
        p = p * s.reshape((-1,) + (1,) * (p.ndim - 1)) + float(m) * coef[:, m]
    return p


def _poly(c, s):
    """Value at s of the polynomial with ascending coefficients c (Horner)."""
    p = c[-1]
    for m in range(len(c) - 2, -1, -1):
        p = p * s + c[m]
    return p


def _poly_d(c, s):
    """Derivative at s of the polynomial with ascending coefficients c."""
    if len(c) < 2:
        return 0.0
    p = (len(c) - 1) * c[-1]
    for m in range(len(c) - 2, 0, -1):
        p = p * s + m * c[m]
    return p


def _divide_out(c, s0):
    """Quotient q of c(s) = (s - s0) q(s) + c(s0), ascending coefficients
    (synthetic division)."""
    K = len(c) - 1
    q = np.zeros(max(K, 1))
    acc = c[K]
    for m in range(K - 1, -1, -1):
        q[m] = acc
        acc = acc * s0 + c[m]
    return q


def real_roots(c):
    """Sorted real roots of the polynomial with ascending coefficients c: the
    eigenvalues of its companion matrix (numpy.roots) whose imaginary part is
    below ROOT_IMAG of their size.  Zero leading coefficients are dropped."""
    c = np.trim_zeros(np.asarray(c, dtype=np.float64), "b")
    if len(c) < 2:
        return np.zeros(0)
    r = np.roots(c[::-1])
    keep = np.abs(r.imag) <= ROOT_IMAG * (1.0 + np.abs(r.real))
    return np.sort(r.real[keep])


def first_exit(c, s0, entry):
    """inf{ s in (s0, 1] : f(s) < 0 } for f the polynomial lambda_i(x(s)) with
    ascending coefficients c, or inf when f stays non-negative.

    entry: face i is the one the path entered through at s0, where f vanishes;
    f is divided by (s - s0) and the quotient (same sign on (s0, 1]) is used.
    The real roots in (s0, 1) cut the interval into pieces of one sign; roots
    within ROOT_MERGE of each other or of the ends count once (a narrower
    excursion is a graze).  The first piece whose middle is negative starts
    the crossing: s0 itself for the first piece, else a root, polished by
    Newton steps that stay between its neighbours."""
    c = np.asarray(c, dtype=np.float64)
    f = _divide_out(c, s0) if entry else c
    pts = [s0]
    for r in real_roots(f):
        if r - pts[-1] > ROOT_MERGE and r < 1.0 - ROOT_MERGE:
            pts.append(float(r))
    pts.append(1.0)
    for k in range(len(pts) - 1):
        mid = 0.5 * (pts[k] + pts[k + 1])
        if _poly(f, mid) < 0.0:
            if k == 0:
                return s0
            r = pts[k]
            lo, hi = 0.5 * (pts[k - 1] + r), mid
            for _ in range(NEWTON_POLISH):
                d = _poly_d(f, r)
                if d == 0.0:
                    break
                rn = r - _poly(f, r) / d
                if not (lo < rn < hi):
                    break
                r = rn
            return r
    return np.inf


def path_coeffs(x, vhist, dt, k):
    """C [n, k+1, 3] of x(s) from x^n and vhist [k, n, 3] (v^n, v^{n-1}, ...)."""
    beta, gam = ab_tables(k)
    n = len(x)
    C = np.zeros((n, k + 1, 3))
    C[:, 0] = x
    for m in range(1, k + 1):
        acc = gam[0][m] * vhist[0]
        for j in range(1, k):
            acc = acc + gam[j][m] * vhist[j]
        C[:, m] = dt * acc
    return C


def lam_coeffs(g, c, C):
    """Coefficients [n, K+1, 4] of lambda_i(x(s)) for the tets' maps g [n,4,3], c [n,4]."""
    K = C.shape[1] - 1
    out = np.zeros((len(C), K + 1, 4))
    for m in range(K + 1):
        for i in range(4):
            v = (g[:, i, 0] * C[:, m, 0] + g[:, i, 1] * C[:, m, 1]) + g[:, i, 2] * C[:, m, 2]
            out[:, m, i] = v + c[:, i] if m == 0 else v
    return out


def _segment_currents(order, A, s0, s1, qw):
    """q w int_{s0}^{s1} W1_j(x(s)) . x'(s) ds for every local j; A are the
    lambda coefficients [n, K+1, 4]."""
    xq, wq = gauss_legendre01_n(2 * order + 2)
    ln = s1 - s0
    spec = basis.w1_spec(order)
    acc = np.zeros((len(A), len(spec)))
    for q in range(len(xq)):
        sq = s0 + ln * xq[q]
        L = _horner(A, sq)
        dL = _horner_deriv(A, sq)
        vals = []
        for (a, b, x, kind) in spec:
            wv = L[:, a] * dL[:, b] - L[:, b] * dL[:, a]
            if kind == "e":
                wv = (3.0 * L[:, x] - 1.0) * wv
            elif kind == "f":
                wv = (3.0 * L[:, x]) * wv
            vals.append(wv)
        acc = acc + wq[q] * np.stack(vals, axis=1)
    return qw * (ln[:, None] * acc)


def _mirror(vec, gw, gg):
    return vec - ((2.0 * geometry.dot3(vec, gw)) / gg)[..., None] * gw


def step(topo, g_all, c_all, x, v, tet, vh, ah, hcount, E, B, q, m, qw, dt, n1, max_cross=4096,
         trace=None, dg_abs=None):
    """One AB step of every particle.

    vh, ah [3, n, 3]: v^{n-1..n-3}, a^{n-1..n-3} (valid: the first hcount);
    E, B gathered at x.  Returns dict with x, v, tet, vh, ah (shifted), dg,
    ncross, hash, status and the order k used.  trace (a list, optional)
    receives one (particle, tet, face, s) per crossing, in walk order;
    dg_abs (optional, [n1]) the sum of the absolute values of the terms added
    into each DOF.
    """
    n = len(x)
    k = min(4, hcount + 1)
    qm = q / m
    a_n = qm * (E + geometry.cross(v, B))
    vhist = np.concatenate([v[None], vh[:k - 1]], axis=0)
    ahist = np.concatenate([a_n[None], ah[:k - 1]], axis=0)
    beta, _ = ab_tables(k)
    acc = beta[0] * ahist[0]
    for j in range(1, k):
        acc = acc + beta[j] * ahist[j]
    v_new = v + dt * acc
    C = path_coeffs(x, vhist, dt, k)
    # history vectors that are mirrored with the path at walls
    vn = v.copy()
    an = a_n.copy()
    vhm = vh.copy()
    ahm = ah.copy()

    T = np.asarray(tet, dtype=np.int64).copy()
    entry = np.full(n, -1, dtype=np.int64)
    s_in = np.zeros(n)
    ncross = np.zeros(n, dtype=np.int64)
    hsh = np.full(n, FNV_OFFSET, dtype=np.uint64)
    status = np.zeros(n, dtype=np.int32)
    dg = np.zeros(n1)
    act = np.arange(n)
    while act.size:
        Ta = T[act]
        A = lam_coeffs(g_all[Ta], c_all[Ta], C[act])
        s0 = s_in[act]
        ent = entry[act]
        found = np.zeros(act.size, dtype=bool)
        best = np.full(act.size, -1, dtype=np.int64)
        s1 = np.ones(act.size)
        for r in range(act.size):
            tbest = np.inf
            for i in range(4):
                ti = first_exit(A[r, :, i], s0[r], ent[r] == i)
                if ti < tbest:                   # strict: ties keep the lowest face
                    tbest, best[r] = ti, i
            if best[r] >= 0:
                found[r] = True
                s1[r] = tbest
        contrib = _segment_currents(topo.order, A, s0, s1, qw)
        np.add.at(dg, topo.dof1[Ta].ravel(), contrib.ravel())
        if dg_abs is not None:
            np.add.at(dg_abs, topo.dof1[Ta].ravel(), np.abs(contrib).ravel())

        go = np.nonzero(found)[0]
        if go.size:
            p = act[go]
            f = best[go]
            if trace is not None:
                trace.extend(zip(p.tolist(), T[p].tolist(), f.tolist(), s1[go].tolist()))
            nb = topo.tet2tet[T[p], f]
            wall = nb < 0
            code = np.where(wall, np.int64(0x80000000) | f, nb).astype(np.uint64)
            hsh[p] = (hsh[p] ^ code) * FNV_PRIME
            ncross[p] += 1
            inner = p[~wall]
            entry[inner] = topo.tet2face[T[inner], f[~wall]]
            T[inner] = nb[~wall]
            s_in[inner] = s1[go][~wall]
            pw = p[wall]
            if pw.size:
                fw = f[wall]
                gw = g_all[T[pw], fw]
                gg = geometry.dot3(gw, gw)
                sw = s1[go][wall]
                hitp = _horner(C[pw], sw)
                C[pw, 0] = hitp + _mirror(C[pw, 0] - hitp, gw, gg)
                for mm in range(1, C.shape[1]):
                    C[pw, mm] = _mirror(C[pw, mm], gw, gg)
                v_new[pw] = _mirror(v_new[pw], gw, gg)
                vn[pw] = _mirror(vn[pw], gw, gg)
                an[pw] = _mirror(an[pw], gw, gg)
                for jj in range(3):
                    vhm[jj, pw] = _mirror(vhm[jj, pw], gw[None][0], gg)
                    ahm[jj, pw] = _mirror(ahm[jj, pw], gw[None][0], gg)
                s_in[pw] = sw
                entry[pw] = fw
            capped = p[ncross[p] >= max_cross]
            status[capped] = 1
            keep = go[ncross[p] < max_cross]
            act = act[keep]
        else:
            act = act[:0]
    x_new = _horner(C, np.ones(n))
    vh_new = np.concatenate([vn[None], vhm[:2]], axis=0)
    ah_new = np.concatenate([an[None], ahm[:2]], axis=0)
    return dict(x=x_new, v=v_new, tet=T, vh=vh_new, ah=ah_new, dg=dg, ncross=ncross, hash=hsh,
                status=status, order=k)

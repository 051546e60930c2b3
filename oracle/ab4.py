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
* Walk: in each tet, lambda_i(x(s)) is a polynomial in s (lambda affine).
  From the entry parameter s0 the interval [s0, 1] is sampled at 8 equal
  steps; in the first step where some lambda_i turns negative, each such face
  gets 8 safeguarded Newton steps inside that bracket (start at its middle;
  the sign of lambda shrinks the bracket; a Newton step that leaves the
  closed bracket is replaced by its middle); the last iterate is the
  crossing.  The
  exit face is the one with the smallest crossing (ties to the lowest index)
  and the particle continues in the neighbour from that parameter.  The entry face counts as 0
  at the entry parameter.  (A grazing excursion shorter than one sample step
  is not split off; charge stays conserved, since the sub-path's ends are in
  the tet and W0 is continuous there.)
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

N_SAMPLES = 8
N_REFINE = 8


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


def step(topo, g_all, c_all, x, v, tet, vh, ah, hcount, E, B, q, m, qw, dt, n1, max_cross=4096):
    """One AB step of every particle.

    vh, ah [3, n, 3]: v^{n-1..n-3}, a^{n-1..n-3} (valid: the first hcount);
    E, B gathered at x.  Returns dict with x, v, tet, vh, ah (shifted), dg,
    ncross, hash, status and the order k used.
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
        span = 1.0 - s0
        prev = _horner(A, s0)
        ent = entry[act]
        for i in range(4):
            prev[ent == i, i] = 0.0
        found = np.zeros(act.size, dtype=bool)
        best = np.full(act.size, -1, dtype=np.int64)
        s1 = np.ones(act.size)
        for j in range(1, N_SAMPLES + 1):
            lo_s = s0 + span * ((j - 1) / N_SAMPLES)
            hi_s = s0 + span * (j / N_SAMPLES)
            cur = _horner(A, hi_s)
            look = ~found
            sbest = np.full(act.size, np.inf)
            for i in range(4):
                cand = look & (cur[:, i] < 0.0)
                if not cand.any():
                    continue
                lo = lo_s.copy()
                hi = hi_s.copy()
                Ai = A[:, :, i:i + 1]
                sx = (lo + hi) * 0.5
                with np.errstate(divide="ignore", invalid="ignore"):
                    for _ in range(N_REFINE):
                        f = _horner(Ai, sx)[:, 0]
                        neg = f < 0.0
                        hi = np.where(neg, sx, hi)
                        lo = np.where(neg, lo, sx)
                        d = _horner_deriv(Ai, sx)[:, 0]
                        sn = sx - f / d
                        ok = (sn >= lo) & (sn <= hi)
                        sx = np.where(ok, sn, (lo + hi) * 0.5)
                upd = cand & (sx < sbest)
                sbest[upd] = sx[upd]
                best[upd] = i
            hit = look & (best >= 0)
            s1[hit] = sbest[hit]
            found |= hit
            prev = cur
        contrib = _segment_currents(topo.order, A, s0, s1, qw)
        np.add.at(dg, topo.dof1[Ta].ravel(), contrib.ravel())

        go = np.nonzero(found)[0]
        if go.size:
            p = act[go]
            f = best[go]
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

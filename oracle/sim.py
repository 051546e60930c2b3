"""One full PIC step of the oracle and its diagnostics.

PIC cycle (Section II, last paragraph; Section III-B): gather E^n, B^n at the
particles, push, walk and deposit Delta g^{n+1} = g^{n+1} - g^n, solve the
Newmark system for e^{n+1}, advance b, measure rho^{n+1}.

Diagnostics (Section IV-D): the continuity residual rho^{n+1} - rho^n -
D^T Delta g^{n+1} on interior W0 DOFs (the paper's "rho vs -[grad] G"), and
the Gauss residual D^T [*eps] e + rho + rho_ion <W0, 1> on interior W0 DOFs
(the paper's "[div] D vs -[grad] G").  The electrostatic start solves the
nodal Laplacian D^T [*eps] D phi = rho + rho_ion <W0,1> with phi = 0 on the
boundary and sets e^0 = e^{-1} = -D phi (the paper is silent on the start).

Several species (the paper's plasma-ball example: ions and electrons) are
advanced one after the other with their own q, m and weight; their currents
and charges add.  Particles are kept concatenated in species order.
Impedance faces (``bface_tag``, see Topology) add [*_I] to the trapezoid
rule (see fields).  Absorbing faces end a particle's path on the wall; the
particle is then re-injected by its species' injector (see inject) before
the charge is measured, so the particle count is constant.
"""

import numpy as np
import scipy.sparse.linalg as spla

from . import ab4, assemble, fields, inject, particles
from .geometry import barycentric_maps
from .topology import Topology


class Sim:
    def __init__(self, xyz, tets, order, q, m, weight, B0=(0.0, 0.0, 0.0),
                 rho_ion=0.0, scheme="trapezoid", gamma=0.5, beta=0.25, matrices=True,
                 max_cross=4096, bface_tag=None, push="boris"):
        self.topo = t = Topology(xyz, tets, order, bface_tag)
        self.g, self.c, self.vol = barycentric_maps(t.xyz, t.tets)
        self.order = order
        self.q, self.m, self.weight = float(q), float(m), float(weight)
        self.qw = self.q * self.weight
        self.B0 = np.asarray(B0, dtype=np.float64)
        self.rho_ion = float(rho_ion)
        self.scheme = scheme
        self.gamma, self.beta = float(gamma), float(beta)
        self.max_cross = max_cross
        if push not in ("boris", "ab4"):
            raise ValueError("push must be 'boris' or 'ab4'")
        self.push = push
        self.hcount = 0
        self.e = np.zeros(t.n1)
        self.e_prev = np.zeros(t.n1)
        self.b = np.zeros(t.n2)
        self.dg_prev = np.zeros(t.n1)
        if matrices:
            self.M = assemble.mass1(t, self.g, self.vol)
            self.K = assemble.curlcurl(t, self.g, self.vol)
            self.C = assemble.curl_matrix(t)
            self.M2 = assemble.mass2(t, self.g, self.vol)
            self.CtM2 = (self.C.T @ self.M2).tocsr()
            self.D = assemble.grad_matrix(t)
            self.load = assemble.nodal_load(t, self.g, self.vol)
            self.I = assemble.impedance(t, self.g)
        self.species = [(self.q, self.m, self.weight)]
        self.offsets = [0]
        self.nstep = 0
        self.injectors = {}
        self.seed = 0
        if push == "ab4" and t.tet_absorb.any():
            raise ValueError("the Adams-Bashforth push has no absorbing walls")

    def set_injection(self, injectors, seed):
        """injectors: list of dicts with species, v_drift[3], v_sigma[3]."""
        self.injectors = {int(d["species"]): (np.asarray(d["v_drift"], dtype=np.float64),
                                              np.asarray(d["v_sigma"], dtype=np.float64)) for d in injectors}
        self.seed = int(seed) & inject.MASK
        self.inj_table = inject.face_table(self.topo)

    # ----------------------------------------------------------------- state
    def set_particles(self, x, v, tet):
        self.x = np.array(x, dtype=np.float64)
        self.v = np.array(v, dtype=np.float64)
        self.tet = np.array(tet, dtype=np.int64)
        self.offsets = [0, len(self.x)]
        self.species = [(self.q, self.m, self.weight)]
        self.rho = self._measure_rho(self.x, self.tet)
        self._reset_history()

    def _reset_history(self):
        """Adams-Bashforth history (v^{n-j}, a^{n-j}, j = 1..3), empty."""
        self.vh = np.zeros((3, len(self.x), 3))
        self.ah = np.zeros((3, len(self.x), 3))
        self.hcount = 0

    def set_species(self, species):
        """species: list of dicts with q, m, weight, x, v, tet."""
        self.species = [(float(s["q"]), float(s["m"]), float(s["weight"])) for s in species]
        self.x = np.concatenate([np.asarray(s["x"], dtype=np.float64).reshape(-1, 3) for s in species])
        self.v = np.concatenate([np.asarray(s["v"], dtype=np.float64).reshape(-1, 3) for s in species])
        self.tet = np.concatenate([np.asarray(s["tet"], dtype=np.int64) for s in species])
        self.offsets = list(np.cumsum([0] + [len(np.asarray(s["tet"])) for s in species]))
        self.rho = self._measure_rho(self.x, self.tet)
        self._reset_history()

    def _slices(self):
        for k, (q, m, w) in enumerate(self.species):
            yield slice(self.offsets[k], self.offsets[k + 1]), q, m, w

    def _measure_rho(self, x, tet):
        """rho of every species; self.rho_abs gets the sums of the absolute
        values of its terms, self.rho_cnt the sums of |q w| of the particles
        that contribute to each DOF."""
        rho = np.zeros(self.topo.n0)
        self.rho_abs = np.zeros(self.topo.n0)
        self.rho_cnt = np.zeros(self.topo.n0)
        for sl, q, m, w in self._slices():
            rho += particles.measure_rho(self.topo, self.g, self.c, x[sl], tet[sl], q * w, self.rho_abs,
                                         self.rho_cnt)
        return rho

    def electrostatic_init(self):
        t = self.topo
        L = (self.D.T @ self.M @ self.D).tocsr()
        src = self.rho + self.rho_ion * self.load
        idx = np.nonzero(t.interior0)[0]
        phi = np.zeros(t.n0)
        if idx.size:
            phi[idx] = spla.spsolve(L[idx][:, idx].tocsc(), src[idx])
        self.e = -(self.D @ phi)
        self.e_prev = self.e.copy()
        return phi

    # ------------------------------------------------------------------ step
    def push_walk(self, dt):
        """Particle half-step of every species; returns the walk record
        (per-particle arrays concatenated in species order, summed current)."""
        t = self.topo
        parts = []
        dg = np.zeros(t.n1)
        dg_abs = np.zeros(t.n1)
        if self.push == "ab4":
            return self._push_walk_ab4(dt)
        for sl, q, m, w in self._slices():
            E, B = particles.gather(t, self.g, self.c, self.e, self.b, self.B0, self.x[sl], self.tet[sl])
            vn = particles.boris(self.v[sl], E, B, q, m, dt)
            x1 = self.x[sl] + dt * vn
            xe, ve, te, d, ncross, hsh, st, ab = particles.walk_deposit(
                t, self.g, self.c, self.x[sl], x1, vn, self.tet[sl], q * w, t.n1, self.max_cross,
                absorb=t.tet_absorb if t.tet_absorb.any() else None, dg_abs=dg_abs)
            dg += d
            k = len(parts)
            if ab.any():
                if k not in self.injectors:
                    raise ValueError("absorbing walls need an injector for every species")
                drift, sigma = self.injectors[k]
                for i in np.nonzero(ab)[0]:
                    xe[i], ve[i], te[i] = inject.sample(self.inj_table, self.seed, self.nstep, sl.start + i,
                                                        drift, sigma)
            parts.append(dict(E=E, B=B, v_half=vn, x_target=x1, x=xe, v=ve, tet=te, ncross=ncross, hash=hsh,
                              status=st, absorbed=ab))
        out = {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}
        out["dg"] = dg
        out["dg_abs"] = dg_abs
        return out

    def _push_walk_ab4(self, dt):
        """Adams-Bashforth step of every species on the quartic path."""
        t = self.topo
        parts = []
        dg = np.zeros(t.n1)
        dg_abs = np.zeros(t.n1)
        for sl, q, m, w in self._slices():
            E, B = particles.gather(t, self.g, self.c, self.e, self.b, self.B0, self.x[sl], self.tet[sl])
            r = ab4.step(t, self.g, self.c, self.x[sl], self.v[sl], self.tet[sl], self.vh[:, sl],
                         self.ah[:, sl], self.hcount, E, B, q, m, q * w, dt, t.n1, self.max_cross,
                         dg_abs=dg_abs)
            dg += r["dg"]
            parts.append(r)
        out = {k: np.concatenate([p[k] for p in parts]) for k in ("x", "v", "tet", "ncross", "hash", "status")}
        out["vh"] = np.concatenate([p["vh"] for p in parts], axis=1)
        out["ah"] = np.concatenate([p["ah"] for p in parts], axis=1)
        out["dg"] = dg
        out["dg_abs"] = dg_abs
        out["order"] = parts[0]["order"] if parts else min(4, self.hcount + 1)
        return out

    def step(self, dt):
        t = self.topo
        w = self.push_walk(dt)
        A = fields.system_matrix(self.M, self.K, dt, self.scheme, self.gamma, self.beta, self.I)
        if self.scheme == "trapezoid":
            r = fields.rhs_trapezoid(self.M, self.K, self.CtM2, self.e, self.b, w["dg"], dt, self.I)
        else:
            r = fields.rhs_wave(self.M, self.K, self.e, self.e_prev, w["dg"], self.dg_prev,
                                dt, self.gamma, self.beta)
        w["rhs"] = r
        e_new = fields.solve(A, r, t.free1)
        b_new = fields.update_b(self.C, self.b, e_new, self.e, dt)
        rho_new = self._measure_rho(w["x"], w["tet"])
        w["continuity"] = (rho_new - self.rho) - self.D.T @ w["dg"]
        w["drho"] = rho_new - self.rho
        self.e_prev, self.e, self.b = self.e, e_new, b_new
        self.dg_prev = w["dg"]
        self.x, self.v, self.tet, self.rho = w["x"], w["v"], w["tet"], rho_new
        if self.push == "ab4":
            self.vh, self.ah = w["vh"], w["ah"]
            self.hcount = min(3, self.hcount + 1)
        self.nstep += 1
        w["gauss"] = self.gauss_residual()
        return w

    def energy(self):
        """W = e.[*eps]e / 2 + b.[*mu^-1]b / 2 (self fields)."""
        return 0.5 * self.e @ (self.M @ self.e) + 0.5 * self.b @ (self.M2 @ self.b)

    def gauss_residual(self):
        return self.D.T @ (self.M @ self.e) + self.rho + self.rho_ion * self.load

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
"""

import numpy as np
import scipy.sparse.linalg as spla

from . import assemble, fields, particles
from .geometry import barycentric_maps
from .topology import Topology


class Sim:
    def __init__(self, xyz, tets, order, q, m, weight, B0=(0.0, 0.0, 0.0),
                 rho_ion=0.0, scheme="trapezoid", gamma=0.5, beta=0.25, matrices=True,
                 max_cross=4096):
        self.topo = t = Topology(xyz, tets, order)
        self.g, self.c, self.vol = barycentric_maps(t.xyz, t.tets)
        self.order = order
        self.q, self.m, self.weight = float(q), float(m), float(weight)
        self.qw = self.q * self.weight
        self.B0 = np.asarray(B0, dtype=np.float64)
        self.rho_ion = float(rho_ion)
        self.scheme = scheme
        self.gamma, self.beta = float(gamma), float(beta)
        self.max_cross = max_cross
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

    # ----------------------------------------------------------------- state
    def set_particles(self, x, v, tet):
        self.x = np.array(x, dtype=np.float64)
        self.v = np.array(v, dtype=np.float64)
        self.tet = np.array(tet, dtype=np.int64)
        self.rho = particles.measure_rho(self.topo, self.g, self.c, self.x, self.tet, self.qw)

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
        """Particle half-step; returns the walk record."""
        t = self.topo
        E, B = particles.gather(t, self.g, self.c, self.e, self.b, self.B0, self.x, self.tet)
        vn = particles.boris(self.v, E, B, self.q, self.m, dt)
        x1 = self.x + dt * vn
        xe, ve, te, dg, ncross, hsh, status = particles.walk_deposit(
            t, self.g, self.c, self.x, x1, vn, self.tet, self.qw, t.n1, self.max_cross)
        return dict(E=E, B=B, v_half=vn, x_target=x1, x=xe, v=ve, tet=te, dg=dg,
                    ncross=ncross, hash=hsh, status=status)

    def step(self, dt):
        t = self.topo
        w = self.push_walk(dt)
        A = fields.system_matrix(self.M, self.K, dt, self.scheme, self.gamma, self.beta)
        if self.scheme == "trapezoid":
            r = fields.rhs_trapezoid(self.M, self.K, self.CtM2, self.e, self.b, w["dg"], dt)
        else:
            r = fields.rhs_wave(self.M, self.K, self.e, self.e_prev, w["dg"], self.dg_prev,
                                dt, self.gamma, self.beta)
        w["rhs"] = r
        e_new = fields.solve(A, r, t.free1)
        b_new = fields.update_b(self.C, self.b, e_new, self.e, dt)
        rho_new = particles.measure_rho(t, self.g, self.c, w["x"], w["tet"], self.qw)
        w["continuity"] = (rho_new - self.rho) - self.D.T @ w["dg"]
        w["drho"] = rho_new - self.rho
        self.e_prev, self.e, self.b = self.e, e_new, b_new
        self.dg_prev = w["dg"]
        self.x, self.v, self.tet, self.rho = w["x"], w["v"], w["tet"], rho_new
        w["gauss"] = self.gauss_residual()
        return w

    def gauss_residual(self):
        return self.D.T @ (self.M @ self.e) + self.rho + self.rho_ion * self.load

"""Newmark field update (Section III-B, eq. maxnmb and the gamma, beta choice).

The printed first-order [b; e] Newmark equation is garbled (an undefined
S_M, forcing at n+1 and n-1 only).  Two readings are implemented:

``trapezoid`` (default; gamma = 1/2, beta = 1/4, "average acceleration"):
the Newmark average-acceleration rule applied to the first-order system
[*eps] e' = C^T [*mu^-1] b - g',  b' = -C e  (Section III-A, eq.
maxwell_semi, with the current entering through G = int J, eq. G/ampere2).
Eliminating b^{n+1} gives one SPD solve per step:

  ([*eps] + dt^2/4 K) e^{n+1} = ([*eps] - dt^2/4 K) e^n + dt C^T [*mu^-1] b^n
                               - (g^{n+1} - g^n),
  b^{n+1} = b^n - dt/2 C (e^{n+1} + e^n),

with K = C^T [*mu^-1] C.  Applying D^T (D^T C^T = 0) leaves
D^T [*eps] (e^{n+1} - e^n) = -D^T (g^{n+1} - g^n): Gauss's law is carried
from step to step for any particle motion (Section III-B, charge conservation
independent of the time stepper), and its null space does not grow
(Section III-C, first sentence).

``wave`` (gamma, beta free; used for the alternative schemes of Section
IV-D: backward difference gamma = 3/2, beta = 1; Galerkin gamma = 3/2,
beta = 0.8): the second-order form [*eps] e'' + K e = -g'' with Newmark
weights
  M (e^{n+1} - 2 e^n + e^{n-1})
   + dt^2 K (beta e^{n+1} + (1/2 + gamma - 2 beta) e^n + (1/2 - gamma + beta) e^{n-1})
   = -(g^{n+1} - 2 g^n + g^{n-1}),
followed by the same trapezoidal b update.

Boundaries: PEC faces (Dirichlet n x E = 0) hold their W1 DOFs at 0.
Impedance faces (first-order absorbing, eq. impedanceBC) add the surface
impedance matrix I = [*_I] to the e row of the first-order system (Section
III-A, the S matrix): [*eps] e' = C^T [*mu^-1] b - I e - g'.  The trapezoid
rule then gives

  ([*eps] + dt^2/4 K + dt/2 I) e^{n+1} = ([*eps] - dt^2/4 K - dt/2 I) e^n
                                         + dt C^T [*mu^-1] b^n - Delta g,

and the discrete energy W = e.[*eps]e/2 + b.[*mu^-1]b/2 drops by exactly
dt ebar.I ebar per step (ebar = (e^{n+1} + e^n)/2) without sources.  The
wave form has no impedance term here.  Linear systems are solved directly
(sparse LU).

Test infrastructure only: part of the CPU oracle, which the product library
never imports.
"""

import numpy as np
import scipy.sparse.linalg as spla


def newmark_coeffs(gamma, beta):
    return beta, 0.5 + gamma - 2.0 * beta, 0.5 - gamma + beta


def system_matrix(M, K, dt, scheme, gamma=0.5, beta=0.25, I=None):
    c1 = 0.25 if scheme == "trapezoid" else newmark_coeffs(gamma, beta)[0]
    A = M + (c1 * dt * dt) * K
    if I is not None and I.nnz:
        if scheme != "trapezoid":
            raise ValueError("impedance boundaries need the trapezoid scheme")
        A = A + (0.5 * dt) * I
    return A.tocsr()


def rhs_trapezoid(M, K, CtM2, e_n, b_n, dg_np1, dt, I=None):
    r = (M @ e_n - (0.25 * dt * dt) * (K @ e_n) + dt * (CtM2 @ b_n)) - dg_np1
    if I is not None and I.nnz:
        r = r - (0.5 * dt) * (I @ e_n)
    return r


def rhs_wave(M, K, e_n, e_nm1, dg_np1, dg_n, dt, gamma, beta):
    _, c2, c3 = newmark_coeffs(gamma, beta)
    return (M @ (2.0 * e_n - e_nm1) - (dt * dt) * (K @ (c2 * e_n + c3 * e_nm1))
            - (dg_np1 - dg_n))


def solve(A, r, free):
    idx = np.nonzero(free)[0]
    out = np.zeros(A.shape[0])
    out[idx] = spla.spsolve(A[idx][:, idx].tocsc(), r[idx])
    return out


def update_b(C, b_n, e_np1, e_n, dt):
    return b_n - (dt * 0.5) * (C @ (e_np1 + e_n))

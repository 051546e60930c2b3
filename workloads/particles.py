"""Seeded particle samplers.

Positions are drawn uniformly inside a set of tets (a tet is picked with
probability proportional to its volume, then a point is drawn uniformly in it
from Dirichlet(1,1,1,1) barycentric weights).  The weights are pulled in by a
relative margin so that every point lies strictly inside the tet it was drawn
in; that tet is returned as the particle's owner.
"""

import numpy as np

from .meshes import tet_volumes


def sample_uniform_in_tets(xyz, tets, n, rng, subset=None, margin=1e-9):
    """Return ``x`` [n,3] float64 and ``owner`` [n] int32."""
    cand = np.arange(len(tets)) if subset is None else np.asarray(subset)
    vol = np.abs(tet_volumes(xyz, tets[cand]))
    owner = cand[rng.choice(len(cand), size=n, p=vol / vol.sum())]
    e = -np.log(rng.uniform(size=(n, 4)))
    lam = e / e.sum(axis=1, keepdims=True)
    lam = lam * (1.0 - 4.0 * margin) + margin
    x = np.einsum("nk,nkd->nd", lam, xyz[tets[owner]])
    return x, owner.astype(np.int32)


def maxwellian(n, vth, rng, drift=(0.0, 0.0, 0.0)):
    """Velocities with independent normal components of std ``vth``."""
    return rng.normal(0.0, vth, size=(n, 3)) + np.asarray(drift, dtype=np.float64)

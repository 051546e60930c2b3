"""Particle injection on tagged boundary faces (test infrastructure: the
oracle of the library's absorbing and injecting walls).

The paper injects its drift-tube beam at one end (Section IV) but says
nothing about how; the reading used here: a particle whose path ends on an
absorbing wall leaves the domain, and its slot is refilled at the end of the
same step by a fresh sample of its species' injector:

* the face is drawn among the injection faces with probability proportional
  to area (faces in global order, areas summed one after the other), the
  point uniformly on that triangle (two uniforms reflected into the lower
  triangle when their sum exceeds 1), the owning tet is the face's tet;
* each velocity component is drift + sigma g with g the Irwin-Hall sum of
  twelve uniforms minus 6 (mean 0, variance 1), so that every step is plain
  arithmetic that both implementations round the same way.

Random numbers come from a counter-based generator: the SplitMix64 output
function (Steele, Lea and Flood, OOPSLA 2014) applied to
seed + (counter + 1) * 0x9E3779B97F4A7C15, i.e. the (counter + 1)-th output
of SplitMix64 seeded with ``seed``; counter = (step << 40) + (particle id << 6)
+ draw.  A uniform is the top 53 bits times 2^-53.
"""

import numpy as np

MASK = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
N_DRAWS = 39  # face, two for the triangle, 36 for the velocity


def splitmix64(seed, counter):
    """The SplitMix64 output for state seed + (counter + 1) * gamma (Python ints)."""
    z = (int(seed) + (int(counter) + 1) * GAMMA) & MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def uniform(seed, counter):
    return (splitmix64(seed, counter) >> 11) * (1.0 / 9007199254740992.0)


def counter(step, pid, draw):
    return ((int(step) << 40) + (int(pid) << 6) + int(draw)) & MASK


def face_table(topo):
    """Injection faces in global face order: vertices [F, 3, 3] (sorted node
    ids), owning tet [F], running area sum [F]."""
    faces = np.nonzero(topo.inject_face & topo.boundary_face)[0]
    verts = topo.xyz[topo.faces[faces]]
    owner = np.full(len(faces), -1, dtype=np.int64)
    where = {int(f): k for k, f in enumerate(faces)}
    for tt in range(topo.n_tets):
        for i in range(4):
            k = where.get(int(topo.tet_faces[tt, i]))
            if k is not None:
                owner[k] = tt
    cum = np.zeros(len(faces))
    run = 0.0
    for k in range(len(faces)):
        a, b, c = verts[k]
        e1 = [b[0] - a[0], b[1] - a[1], b[2] - a[2]]
        e2 = [c[0] - a[0], c[1] - a[1], c[2] - a[2]]
        cx = e1[1] * e2[2] - e1[2] * e2[1]
        cy = e1[2] * e2[0] - e1[0] * e2[2]
        cz = e1[0] * e2[1] - e1[1] * e2[0]
        area = 0.5 * float(np.sqrt((cx * cx + cy * cy) + cz * cz))
        run = run + area
        cum[k] = run
    return verts, owner, cum


def sample(table, seed, step, pid, drift, sigma):
    """One injected particle: (x[3], v[3], tet)."""
    verts, owner, cum = table
    u = [uniform(seed, counter(step, pid, d)) for d in range(N_DRAWS)]
    target = u[0] * cum[-1]
    k = min(int(np.searchsorted(cum, target, side="right")), len(cum) - 1)
    a, b, c = verts[k]
    u1, u2 = u[1], u[2]
    if u1 + u2 > 1.0:
        u1, u2 = 1.0 - u1, 1.0 - u2
    x = np.array([(a[j] + u1 * (b[j] - a[j])) + u2 * (c[j] - a[j]) for j in range(3)])
    v = np.zeros(3)
    for j in range(3):
        g = 0.0
        for m in range(12):
            g = g + u[3 + 12 * j + m]
        v[j] = drift[j] + sigma[j] * (g - 6.0)
    return x, v, int(owner[k])

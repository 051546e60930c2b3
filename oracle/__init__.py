"""Plain FP64 CPU oracle of the higher-order charge-conserving EM-FEMPIC step.

TEST INFRASTRUCTURE ONLY.  Nothing in the product library imports, links or
runs this package; only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may use it.  It shares no code with the CUDA
library: it is written from the paper's definitions (Crawford et al.,
"Higher Order Charge Conserving Electromagnetic Finite Element Particle in
Cell Method", arXiv 2111.12411) with numpy/scipy as the only helpers.

Modules (each function cites the passage it follows):

* ``topology``  - mesh complex {N, E, F, T}, canonical entity and DOF numbering
  (Section III-A).
* ``geometry``  - barycentric maps of the tets.
* ``basis``     - interpolatory Whitney bases W0, W1, W2 of order 1 and 2
  (Appendix), their gradients/curls.
* ``quadrature`` - Gauss-Legendre rules on [0,1] and a collapsed-cube rule on
  the tetrahedron.
* ``assemble``  - Hodge matrices, curl-curl matrix, exact-sequence maps D, C,
  nodal Laplacian (Section III-A).
* ``particles`` - field gather, Lorentz push, tet walk and the path-integral
  current deposit (Section III-B), charge measurement with W0.
* ``fields``    - Newmark update of the fields (Section III-B, eq. maxnmb).
* ``sim``       - one full PIC step and diagnostics (Section IV-D).
"""

from . import topology, geometry, basis, quadrature, assemble, particles, fields, sim  # noqa: F401

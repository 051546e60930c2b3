"""Seeded synthetic inputs for the EM-FEMPIC particle loop.

This package only *generates inputs*: tetrahedral meshes (node coordinates and
tet connectivity), particle positions/velocities with their owning tet, and
random field-state vectors for single-step comparisons.  It holds none of the
method's arithmetic (no basis functions, no matrices, no push, no walk), so the
CUDA library and the CPU oracle can both be fed from it without sharing code.
"""

from .meshes import kuhn_box, polar_tube, tet_volumes, tube_wall_tags  # noqa: F401
from .particles import sample_uniform_in_tets, maxwellian  # noqa: F401
from .configs import make_config, make_batch, make_requests, build_request, random_dof_vector, CONFIG_NAMES  # noqa: F401

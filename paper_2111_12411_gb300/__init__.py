"""GB300-native EM-FEMPIC: the higher-order charge-conserving finite-element
particle-in-cell step (arXiv 2111.12411) as hand-written sm_103a CUDA kernels
behind a C ABI (``include/fempic.h``).

The native library is loaded lazily by ``native.load()``; there is no CPU
fallback.  ``build.build()`` compiles it in-tree.
"""

from .native import (Simulation, Batch, FemPICError, load,  # noqa: F401
                     femPIC_create, femPIC_step, femPIC_step_async, femPIC_sync, femPIC_get,
                     femPIC_set, femPIC_get_device, femPIC_set_device, femPIC_apply,
                     femPIC_eval_fields, femPIC_get_info, femPIC_last_timing, femPIC_destroy,
                     femPIC_last_error, femPIC_batch_create, femPIC_batch_step,
                     femPIC_batch_timing, femPIC_batch_destroy, femPIC_batch_last_error)
from .metrics import StepLog, run_logged  # noqa: F401,E402

"""Per-step metrics as JSON lines.

One object per step: the step index, the device diagnostics (continuity and
Gauss residuals with their reference norms, the div b moments, face
crossings, absorbed particles, CG iterations and residual, as the library
reports them in femPIC_diag) and the device times of the step's phases
(femPIC_last_timing).  The paper's own accuracy figures are these residuals;
the run's throughput follows from the times.
"""

import json
import math


def _clean(v):
    """JSON has no NaN or infinity: write them as null."""
    if isinstance(v, float) and not math.isfinite(v):
        return None
    return v


class StepLog:
    """Append one JSON line per recorded step to a file path or an open text file."""

    def __init__(self, target):
        self._own = isinstance(target, str)
        self.f = open(target, "a") if self._own else target
        self.lines = 0

    def record(self, step, diag=None, timing=None, **extra):
        row = {"step": int(step)}
        for name, d in (("diag", diag), ("timing_ms", timing)):
            if d:
                row[name] = {k: _clean(float(v)) for k, v in d.items()}
        row.update({k: _clean(v) for k, v in extra.items()})
        self.f.write(json.dumps(row) + "\n")
        self.lines += 1

    def close(self):
        self.f.flush()
        if self._own:
            self.f.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def run_logged(sim, dt, n_steps, log, every=1, first_step=0):
    """Advance ``sim`` by n_steps steps of dt, one call per step, recording
    every ``every``-th step and the last one.  The residual norms are those
    of a handle created with diagnostics on (zero otherwise); the times are
    the device times of the recorded step alone."""
    for k in range(n_steps):
        sim.step(dt)
        if (k + 1) % every == 0 or k + 1 == n_steps:
            log.record(first_step + k + 1, sim.diag(), sim.last_timing())
    return log.lines

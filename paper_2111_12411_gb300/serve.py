"""Serving many EM-FEMPIC simulations on one GPU with continuous batching.

The paper runs one simulation at a time; this runtime keeps many independent
simulations (different meshes, orders and particle counts) resident in HBM
and advances them together:

* requests arrive over time (``arrival`` seconds after the server starts);
* a request is admitted when its estimated device footprint fits the HBM
  budget and a slot is free; its mesh, DOFs and particles are uploaded once
  (``femPIC_create``) and stay on the device until it finishes;
* all admitted requests advance together, one chunk of ``chunk_steps`` steps
  at a time, through one batch (one launch per kernel for all of them);
  requests that arrived meanwhile join at the next chunk boundary, so new
  work overlaps with work already on the GPU (continuous batching);
* a request that has run its chunks returns its result (positions, field DOFs,
  charge) and frees its memory, which admits the next ones.

The latency of every chunk of every request and the aggregate particle-steps
per second are recorded; ``Server.report()`` gives p50/p99 chunk latency.
"""

import time

import numpy as np

from .native import Batch, Simulation


def estimate_device_bytes(n_tets, order, n_particles):
    """Device footprint model: per-particle state (positions, velocities,
    their sort double buffers and staging, ids, crossing records: 148 B) plus
    per-tet mesh, DOF maps, CSR matrices and field vectors (measured for the
    Kuhn box meshes: about 2.3 kB per tet at order 1 and 13 kB at order 2)."""
    per_tet = 2300 if order == 1 else 13000
    return int(148 * n_particles + per_tet * n_tets + (8 << 20))


class Request:
    def __init__(self, rid, cfg, arrival, n_chunks, chunk_steps):
        if int(n_chunks) < 1 or int(chunk_steps) < 1:
            raise ValueError(f"request {rid}: n_chunks and chunk_steps must be at least 1")
        self.id = rid
        self.cfg = cfg
        self.arrival = arrival
        self.n_chunks = n_chunks
        self.chunk_steps = chunk_steps
        self.sim = None
        self.done_chunks = 0
        self.steps_done = 0
        self.steps_in_chunk = 0  # steps of the current chunk taken so far
        self.chunk_time = 0.0    # and their device-synchronised wall time
        self.admitted_at = None
        self.finished_at = None
        self.chunk_latency = []
        self.result = None
        self.bytes = estimate_device_bytes(len(cfg["tets"]), cfg["order"], len(cfg["x"]))


class Server:
    def __init__(self, hbm_budget_bytes, max_slots=64, device=0, precision=None,
                 result_keys=("X", "E", "RHO"), clock=time.perf_counter, sleep=time.sleep,
                 make_sim=None, make_batch=None):
        """make_sim(cfg, **kw) and make_batch(sims) default to
        Simulation.from_config and Batch; clock and sleep to the wall clock."""
        self.make_sim = make_sim or Simulation.from_config
        self.make_batch = make_batch or Batch
        self.sleep = sleep
        self.budget = int(hbm_budget_bytes)
        self.max_slots = max_slots
        self.device = device
        self.precision = precision
        self.result_keys = result_keys
        self.clock = clock
        self.waiting = []
        self.active = []
        self.finished = []
        self.used = 0
        self.batch = None
        self.batch_members = None
        self.particle_steps = 0
        self.busy_s = 0.0
        self.t0 = None

    def submit(self, req):
        if req.bytes > self.budget:
            raise ValueError(f"request {req.id} needs about {req.bytes} bytes, more than the HBM budget")
        self.waiting.append(req)
        self.waiting.sort(key=lambda r: r.arrival)

    # -------------------------------------------------------------- admission
    def _admit(self, now):
        admitted = False
        keep = []
        for r in self.waiting:
            if (r.arrival <= now and len(self.active) < self.max_slots
                    and self.used + r.bytes <= self.budget):
                kw = {"device": self.device}
                if self.precision:
                    kw["precision"] = self.precision
                r.sim = self.make_sim(r.cfg, **kw)
                real = int(r.sim.info.device_bytes)
                r.bytes = max(r.bytes, real)
                self.used += r.bytes
                r.admitted_at = self.clock() - self.t0
                self.active.append(r)
                admitted = True
            else:
                keep.append(r)
        self.waiting = keep
        return admitted

    def _retire(self):
        still = []
        for r in self.active:
            if r.steps_done >= r.n_chunks * r.chunk_steps:
                r.result = {k: r.sim.get(k) for k in self.result_keys}
                r.sim.close()
                r.sim = None
                self.used -= r.bytes
                r.finished_at = self.clock() - self.t0
                self.finished.append(r)
            else:
                still.append(r)
        changed = len(still) != len(self.active)
        self.active = still
        return changed

    # ------------------------------------------------------------------- loop
    def run(self, max_wall_s=None):
        """Serve until every submitted request has finished."""
        self.t0 = self.clock()
        while self.waiting or self.active:
            now = self.clock() - self.t0
            if max_wall_s is not None and now > max_wall_s:
                break
            changed = self._admit(now)
            if not self.active:
                nxt = min(r.arrival for r in self.waiting)
                if self.used == 0 and all(r.bytes > self.budget for r in self.waiting):
                    raise RuntimeError("a request does not fit the HBM budget")
                self.sleep(max(0.0, min(0.05, nxt - now)))
                continue
            members = [r.sim for r in self.active]
            if changed or self.batch is None or self.batch_members != [id(s) for s in members]:
                if self.batch is not None:
                    self.batch.close()
                self.batch = self.make_batch(members)
                self.batch_members = [id(s) for s in members]
            # advance to the nearest chunk boundary among the active requests,
            # where the ones that arrived meanwhile can join
            steps = min(r.chunk_steps - r.steps_in_chunk for r in self.active)
            dts = np.array([r.cfg["dt"] for r in self.active])
            t_a = self.clock()
            self.batch.step(dts, steps)
            dt_run = self.clock() - t_a
            self.busy_s += dt_run
            for r in self.active:
                r.steps_done += steps
                r.steps_in_chunk += steps
                r.chunk_time += dt_run
                if r.steps_in_chunk == r.chunk_steps:
                    r.chunk_latency.append(r.chunk_time)
                    r.done_chunks += 1
                    r.steps_in_chunk = 0
                    r.chunk_time = 0.0
                self.particle_steps += steps * r.sim.n_particles
            if self._retire() and self.batch is not None:
                self.batch.close()
                self.batch = None
        if self.batch is not None:
            self.batch.close()
            self.batch = None
        return self.finished

    def report(self):
        lat = np.array([x for r in self.finished for x in r.chunk_latency])
        wall = self.clock() - self.t0 if self.t0 is not None else 0.0
        return {
            "requests": len(self.finished),
            "chunks": int(lat.size),
            "p50_chunk_latency_s": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_chunk_latency_s": float(np.percentile(lat, 99)) if lat.size else None,
            "particle_steps_per_s_busy": self.particle_steps / self.busy_s if self.busy_s else None,
            "particle_steps_per_s_wall": self.particle_steps / wall if wall else None,
            "wall_s": wall,
            "busy_s": self.busy_s,
            "mean_queue_wait_s": float(np.mean([r.admitted_at - r.arrival for r in self.finished]))
            if self.finished else None,
        }

"""The serving runtime's host logic on the CPU, with stand-ins for the
library's simulations and batch and a simulated clock: admission by HBM
budget and free slots, late arrivals joining at chunk boundaries
(continuous batching), every request advanced by exactly its own
n_chunks x chunk_steps steps even when chunk sizes differ, memory returned on
retirement, and an oversize request refused at submission."""

import types

import numpy as np
import pytest

from paper_2111_12411_gb300.serve import Request, Server, estimate_device_bytes


class World:
    def __init__(self):
        self.t = 0.0
        self.batches = []
        self.used_seen = []
        self.server = None

    def clock(self):
        return self.t

    def sleep(self, d):
        self.t += max(d, 1e-3)

    def make_sim(self, cfg, **kw):
        sim = types.SimpleNamespace(cfg=cfg, steps=0, closed=False, n_particles=len(cfg["x"]),
                                    info=types.SimpleNamespace(device_bytes=cfg["real_bytes"]))
        sim.get = lambda k: {"STEPS": sim.steps}[k]
        sim.close = lambda: setattr(sim, "closed", True)
        return sim

    def make_batch(self, sims):
        world = self
        ids = [s.cfg["id"] for s in sims]
        self.batches.append(ids)

        class B:
            def step(self, dts, n):
                assert len(dts) == len(sims) and n >= 1
                assert not any(s.closed for s in sims)
                world.t += 0.01 * n
                world.used_seen.append((world.server.used, len(sims)))
                for s in sims:
                    s.steps += n

            def close(self):
                pass
        return B()


def _cfg(i, n_tets, n_part, order=1, real_bytes=None):
    cfg = {"id": i, "tets": np.zeros((n_tets, 4), np.int32), "x": np.zeros((n_part, 3)), "order": order,
           "dt": 1e-12 * (i + 1)}
    cfg["real_bytes"] = real_bytes if real_bytes is not None else estimate_device_bytes(n_tets, order, n_part)
    return cfg


def test_admission_budget_slots_and_exact_steps():
    w = World()
    rng = np.random.default_rng(3)
    per = estimate_device_bytes(1000, 1, 5000)
    budget = 3 * per + per // 2  # room for three requests at a time
    srv = Server(budget, max_slots=4, clock=w.clock, sleep=w.sleep, make_sim=w.make_sim,
                 make_batch=w.make_batch, result_keys=("STEPS",))
    w.server = srv
    reqs = []
    for i in range(9):
        r = Request(i, _cfg(i, 1000, 5000), arrival=0.02 * i, n_chunks=int(rng.integers(1, 4)),
                    chunk_steps=int(rng.choice([2, 3, 5])))
        reqs.append(r)
        srv.submit(r)
    done = srv.run()
    assert len(done) == 9 and srv.used == 0 and not srv.active and not srv.waiting
    for r in reqs:
        assert r.result["STEPS"] == r.n_chunks * r.chunk_steps
        assert len(r.chunk_latency) == r.n_chunks and all(x > 0 for x in r.chunk_latency)
        assert r.admitted_at >= r.arrival and r.finished_at > r.admitted_at
    assert all(u <= budget and n <= 3 for u, n in w.used_seen)
    assert max(n for _, n in w.used_seen) == 3
    # continuous batching: some request joined a batch while another was mid-run
    joined = any(set(a) & set(b) and set(b) - set(a) for a, b in zip(w.batches, w.batches[1:]))
    assert joined
    rep = srv.report()
    assert rep["requests"] == 9 and rep["chunks"] == sum(r.n_chunks for r in reqs)
    assert rep["p99_chunk_latency_s"] >= rep["p50_chunk_latency_s"] > 0


def test_slot_limit_and_late_arrival():
    w = World()
    srv = Server(1 << 40, max_slots=2, clock=w.clock, sleep=w.sleep, make_sim=w.make_sim,
                 make_batch=w.make_batch, result_keys=("STEPS",))
    w.server = srv
    reqs = [Request(0, _cfg(0, 10, 10), 0.0, 3, 4), Request(1, _cfg(1, 10, 10), 0.0, 1, 4),
            Request(2, _cfg(2, 10, 10), 0.0, 1, 4), Request(3, _cfg(3, 10, 10), 5.0, 2, 1)]
    for r in reqs:
        srv.submit(r)
    srv.run()
    assert max(n for _, n in w.used_seen) == 2
    assert reqs[2].admitted_at >= reqs[1].finished_at  # waited for a slot
    assert reqs[3].admitted_at >= 5.0                  # not before it arrived
    assert [r.result["STEPS"] for r in reqs] == [12, 4, 4, 2]


def test_oversize_or_empty_request_refused():
    srv = Server(1 << 20)
    with pytest.raises(ValueError):
        srv.submit(Request(0, _cfg(0, 100000, 10), 0.0, 1, 1))
    with pytest.raises(ValueError):
        Request(1, _cfg(1, 10, 10), 0.0, 0, 5)
    with pytest.raises(ValueError):
        Request(2, _cfg(2, 10, 10), 0.0, 2, 0)

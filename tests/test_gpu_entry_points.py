"""GPU tests of the entry points and detectors that take device buffers or
need a test build of the library.

* femPIC_get_device / femPIC_set_device: every quantity read into a device
  buffer equals femPIC_get's host copy; state loaded from device buffers
  gives the same next step (strict mode, bit-exact) as the same state loaded
  from host buffers.
* femPIC_set from host buffers refuses non-finite X or V and out-of-range
  tet ids (checked on the device after the staging copy) and leaves the
  particle state untouched.
* The bounds-checked build (-DFEMPIC_CHECKS=1): an out-of-range tet id handed
  over through femPIC_set_device is refused with FEMPIC_ERR_BOUNDS before it
  is copied or read; the handle keeps working with valid ids.
* The grid barrier's bounded wait: a test build in which one CTA of the
  persistent CG never arrives (and the spin limit is short) makes the other
  CTAs' waits run out; the step returns FEMPIC_ERR_BARRIER and the context
  stays usable (no fault, no hang).

The two test builds run in child processes (FEMPIC_LIB selects the library).
"""

import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

import workloads
from gpu_helpers import build_lib

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def lib():
    return build_lib()


def test_device_buffer_transfers_round_trip():
    import torch
    from paper_2111_12411_gb300 import Simulation, native
    cfg = workloads.make_config(0, n_particles=5003)
    a = Simulation.from_config(cfg, precision="fp64_strict", diagnostics=True)
    a.step(cfg["dt"], 2)
    dev = torch.device("cuda", 0)
    for q in ("E", "E_PREV", "B", "DG", "DG_PREV", "RHO", "X", "V", "TET", "NCROSS", "HASH"):
        host = a.get(q)
        buf = torch.empty(host.nbytes, dtype=torch.uint8, device=dev)
        native.femPIC_get_device(a.h, q, buf.data_ptr(), host.nbytes)
        torch.cuda.synchronize()
        got = buf.cpu().numpy().view(host.dtype).reshape(host.shape)
        assert np.array_equal(got, host), q
    state = {q: a.get(q) for q in ("E", "E_PREV", "B", "DG", "DG_PREV", "X", "V", "TET")}
    b = Simulation.from_config(cfg, precision="fp64_strict", es_init=False)
    c = Simulation.from_config(cfg, precision="fp64_strict", es_init=False)
    for q, v in state.items():
        b.set(q, v)
        t = torch.from_numpy(np.ascontiguousarray(v).view(np.uint8).reshape(-1).copy()).to(dev)
        native.femPIC_set_device(c.h, q, t.data_ptr(), v.nbytes)
        torch.cuda.synchronize()
    for q, v in state.items():
        assert np.array_equal(c.get(q), v), q
    b.step(cfg["dt"])
    c.step(cfg["dt"])
    for q in ("X", "V", "TET", "HASH"):
        assert np.array_equal(c.get(q), b.get(q)), q
    assert np.array_equal(c.get("E"), b.get("E")) or np.linalg.norm(c.get("E") - b.get("E")) <= \
        1e-9 * np.linalg.norm(b.get("E"))
    with pytest.raises(native.FemPICError) as ei:  # a short buffer is refused
        native.femPIC_set_device(c.h, "X", t.data_ptr(), 8)
    assert ei.value.code == native.FEMPIC_ERR_SIZE
    for s in (a, b, c):
        s.close()


def test_host_set_refuses_bad_particle_state():
    """femPIC_set validates host X, V and TET on the device after the staging
    copy: a non-finite value or a tet id outside [0, n_tets) is refused with
    FEMPIC_ERR_ARG naming the first bad particle, and nothing of it reaches
    the particle state (X, V, TET and the measured RHO unchanged, the next
    step bit-identical to a handle that saw no refused call)."""
    from paper_2111_12411_gb300 import Simulation, native
    cfg = workloads.make_config(0, n_particles=5003)
    a = Simulation.from_config(cfg, precision="fp64_strict", es_init=False)
    b = Simulation.from_config(cfg, precision="fp64_strict", es_init=False)
    a.step(cfg["dt"])
    b.step(cfg["dt"])
    before = {q: a.get(q) for q in ("X", "V", "TET", "RHO")}
    n_tets = a.info.n_tets
    cases = []
    for q, val in (("X", np.nan), ("X", np.inf), ("V", -np.inf), ("V", np.nan)):
        for p in (0, 2711, a.n_particles - 1):
            cases.append((q, p, val))
    for val in (-1, n_tets, np.iinfo(np.int32).min):
        for p in (0, 4999):
            cases.append(("TET", p, val))
    for q, p, val in cases:
        bad = before[q].copy()
        bad[p] = val
        if q != "TET":
            bad[p + 1:] = np.nan  # later bad elements: the first is named
        with pytest.raises(native.FemPICError) as ei:
            a.set(q, bad)
        assert ei.value.code == native.FEMPIC_ERR_ARG, (q, p)
        assert f"particle {p}" in str(ei.value), (q, p, str(ei.value))
        for k, v in before.items():
            assert np.array_equal(a.get(k), v), (q, p, k)
    # a valid set after the refusals is taken; the field state is copied from
    # one handle to both (each handle's own first step summed its deposit with
    # FP64 atomics, in an order that may differ in the last bits)
    state = {q: a.get(q) for q in ("E", "E_PREV", "B", "DG", "DG_PREV")}
    state.update({q: before[q] for q in ("X", "V", "TET")})
    for q, v in state.items():
        a.set(q, v)
        b.set(q, v)
    a.step(cfg["dt"])
    b.step(cfg["dt"])
    for q in ("X", "V", "TET", "HASH"):
        assert np.array_equal(a.get(q), b.get(q)), q
    a.close()
    b.close()


def _child(variant, body):
    from paper_2111_12411_gb300 import build
    path = build.build(variant=variant)
    env = dict(os.environ, FEMPIC_LIB=path, PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    script = "import sys\nsys.path.insert(0, %r)\n" % ROOT + textwrap.dedent(body)
    p = subprocess.run([sys.executable, "-c", script], env=env, capture_output=True, text=True, timeout=600,
                       cwd=ROOT)
    assert p.returncode == 0, p.stdout + p.stderr
    return p.stdout


def test_checked_build_refuses_out_of_range_tet_ids():
    out = _child("checked", """
        import numpy as np, torch, workloads
        from paper_2111_12411_gb300 import Simulation, native
        assert native.load()._name.endswith("libfempic_checked.so")
        cfg = workloads.make_config(0, n_particles=3001)
        g = Simulation.from_config(cfg, diagnostics=True)
        g.step(cfg["dt"])
        tet = g.get("TET")
        bad = tet.copy()
        bad[1234] = g.info.n_tets + 5
        t = torch.from_numpy(bad).cuda()
        try:
            native.femPIC_set_device(g.h, "TET", t.data_ptr(), bad.nbytes)
            raise SystemExit("out-of-range tet id accepted")
        except native.FemPICError as e:
            assert e.code == native.FEMPIC_ERR_BOUNDS, e
        assert np.array_equal(g.get("TET"), tet)      # nothing was copied
        t = torch.from_numpy(tet).cuda()
        native.femPIC_set_device(g.h, "TET", t.data_ptr(), tet.nbytes)
        g.step(cfg["dt"])
        d = g.diag()
        assert d["status"] == 0 and d["continuity_abs"] <= 1e-12 * d["continuity_ref"]
        g.close()
        print("checked ok")
    """)
    assert "checked ok" in out


def test_barrier_wait_runs_out_and_reports():
    out = _child("barrier_test", """
        import time
        import numpy as np, workloads
        from paper_2111_12411_gb300 import Simulation, native
        assert native.load()._name.endswith("libfempic_barrier_test.so")
        cfg = workloads.make_config(0, n_particles=2000)
        g = Simulation.from_config(cfg, es_init=False)
        t0 = time.perf_counter()
        try:
            g.step(cfg["dt"])
            raise SystemExit("the step returned without the barrier error")
        except native.FemPICError as e:
            assert e.code == native.FEMPIC_ERR_BARRIER, e
        dt = time.perf_counter() - t0
        x = g.get("X")                                 # the context is still usable
        assert x.shape == (2000, 3) and np.isfinite(x).all()
        g.close()
        print(f"barrier ok {dt:.2f} s")
    """)
    assert "barrier ok" in out

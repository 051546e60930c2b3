"""Per-step JSON-lines metrics (host logic, CPU): one parseable object per
recorded step with the diagnostics and phase times it was given, non-finite
values written as null, the recording period honoured and the last step
always written."""

import io
import json

from paper_2111_12411_gb300.metrics import StepLog, run_logged


class FakeSim:
    def __init__(self):
        self.n = 0

    def step(self, dt):
        self.n += 1

    def diag(self):
        return {"continuity_abs": 1e-20 * self.n, "continuity_ref": 1.0, "cg_iterations": 170 + self.n,
                "gauss_abs": float("nan")}

    def last_timing(self):
        return {"particle_ms": 1.3, "field_ms": 64.6}


def test_run_logged_writes_one_line_per_recorded_step():
    buf = io.StringIO()
    log = StepLog(buf)
    assert run_logged(FakeSim(), 1e-11, 7, log, every=3) == 3
    rows = [json.loads(line) for line in buf.getvalue().splitlines()]
    assert [r["step"] for r in rows] == [3, 6, 7]
    assert rows[0]["diag"]["cg_iterations"] == 173.0 and rows[2]["diag"]["continuity_abs"] == 7e-20
    assert rows[1]["diag"]["gauss_abs"] is None
    assert rows[2]["timing_ms"] == {"particle_ms": 1.3, "field_ms": 64.6}


def test_step_log_to_path(tmp_path):
    p = tmp_path / "steps.jsonl"
    with StepLog(str(p)) as log:
        log.record(1, {"absorbed": 4181.0}, None, chunk_latency_s=0.25)
        log.record(2)
    rows = [json.loads(line) for line in p.read_text().splitlines()]
    assert rows == [{"step": 1, "diag": {"absorbed": 4181.0}, "chunk_latency_s": 0.25}, {"step": 2}]

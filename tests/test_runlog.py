"""Run logs (host logic, a fake engine): reports at the interval and at the
end, force checks at multiples of their interval, records that read back."""

import numpy as np
import pytest

from paper_1311_3890_b300.runlog import RunLog, read_log, run_logged
from paper_1311_3890_b300.tbsma import FCheckC, ObsC


class FakeEngine:
    def __init__(self, W=3):
        self.W, self.t, self.checks = W, 0, []

    def step(self, n, dt):
        assert dt == 2.0
        self.t += n

    def observables(self):
        ob = np.ctypeslib.as_array((ObsC * self.W)()).copy()
        ob["step"] = self.t
        ob["strain"] = 1e-6 * self.t * (1 + np.arange(self.W))
        ob["n_rebuilds"] = self.t // 100
        return ob

    def step_observe(self, n, dt):
        self.step(n, dt)
        return self.observables()

    def force_check(self):
        self.checks.append(self.t)
        fc = np.ctypeslib.as_array((FCheckC * self.W)()).copy()
        fc["norm_err"] = 4e-6
        return fc


def test_reports_and_checks(tmp_path):
    eng = FakeEngine()
    path = str(tmp_path / "run.jsonl")
    with RunLog(path, workload="test", wires=3) as log:
        last = run_logged(eng, 2500, log, report_every=1000, check_every=2000)
    recs = read_log(path)
    assert recs[0] == {"kind": "run", "workload": "test", "wires": 3}
    reports = [r for r in recs if r["kind"] == "report"]
    assert [r["step"] for r in reports] == [1000, 2000, 2500]
    assert reports[-1]["strain"] == pytest.approx([2.5e-3, 5e-3, 7.5e-3])
    assert reports[-1]["n_rebuilds"] == [25, 25, 25] and isinstance(reports[-1]["n_rebuilds"][0], int)
    checks = [r for r in recs if r["kind"] == "force_check"]
    assert [r["step"] for r in checks] == [2000] and eng.checks == [2000]
    assert checks[0]["norm_err"] == [4e-6] * 3
    assert int(last["step"][0]) == 2500


def test_zero_steps_still_reports(tmp_path):
    eng = FakeEngine(1)
    with RunLog(str(tmp_path / "r.jsonl")) as log:
        run_logged(eng, 0, log, check_every=0)
    recs = read_log(str(tmp_path / "r.jsonl"))
    assert [r["kind"] for r in recs] == ["run", "report"] and recs[1]["step"] == 0


def test_bad_arguments(tmp_path):
    with RunLog(str(tmp_path / "r.jsonl")) as log:
        with pytest.raises(ValueError):
            run_logged(FakeEngine(), 10, log, report_every=0)

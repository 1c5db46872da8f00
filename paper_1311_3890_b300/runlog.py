"""Run logs of a batched MD run as JSON lines.

A long run reports every wire's observables at a fixed interval (Eq. 4-5:
strain, stress, energies, temperature, plus the rebuild count and status
word) and checks the mixed-precision forces against the FP64 passes at
another (the force-error gate).  `run_logged` steps an Engine and writes
both to a RunLog; `read_log` returns the records.  One record per line:

    {"kind": "run", ...caller's metadata}
    {"kind": "report", "step": s, "<field>": [per-wire values], ...}
    {"kind": "force_check", "step": s, "max_err_scaled": [...], "norm_err": [...], ...}
"""

from __future__ import annotations

import json

import numpy as np

REPORT_FIELDS = ("strain", "e_pot", "e_kin", "temp", "sigma_xx", "virial_xx", "n_rebuilds",
                 "status")
CHECK_FIELDS = ("max_err_scaled", "max_err_raw", "norm_err", "max_abs_err")


def _values(a: np.ndarray) -> list:
    return [int(v) if np.issubdtype(a.dtype, np.integer) else float(v) for v in a]


class RunLog:
    """Append-only JSON-lines log; usable as a context manager."""

    def __init__(self, path: str, **meta):
        self.path = path
        self.f = open(path, "w")
        self._write({"kind": "run", **meta})

    def _write(self, rec: dict) -> None:
        self.f.write(json.dumps(rec) + "\n")
        self.f.flush()

    def report(self, ob: np.ndarray) -> None:
        """One record of Engine.observables() (a structured array over wires)."""
        steps = np.unique(ob["step"])
        if steps.size != 1:
            raise ValueError("the wires of one report must share the step")
        rec = {"kind": "report", "step": int(steps[0])}
        for k in REPORT_FIELDS:
            rec[k] = _values(np.asarray(ob[k]))
        self._write(rec)

    def force_check(self, step: int, fc: np.ndarray) -> None:
        """One record of Engine.force_check() at `step`."""
        rec = {"kind": "force_check", "step": int(step)}
        for k in CHECK_FIELDS:
            rec[k] = _values(np.asarray(fc[k]))
        self._write(rec)

    def close(self) -> None:
        if not self.f.closed:
            self.f.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def run_logged(eng, n_steps: int, log: RunLog, dt: float = 2.0, report_every: int = 1000,
               check_every: int = 1000) -> np.ndarray:
    """Advance `eng` by n_steps, reporting every `report_every` steps (and at
    the end) and force-checking at every report whose step is a multiple of
    `check_every` (0: never).  Returns the last report."""
    if report_every < 1 or n_steps < 0 or check_every < 0:
        raise ValueError("report_every >= 1, n_steps >= 0 and check_every >= 0")
    done, ob = 0, None
    while done < n_steps or ob is None:
        k = min(report_every, n_steps - done)
        if k > 0:  # the steps and their report in one call
            ob = eng.step_observe(k, dt)
            done += k
        else:
            ob = eng.observables()
        log.report(ob)
        step = int(ob["step"][0])
        if check_every and step % check_every == 0:
            log.force_check(step, eng.force_check())
    return ob


def read_log(path: str) -> list[dict]:
    with open(path) as f:
        return [json.loads(line) for line in f if line.strip()]

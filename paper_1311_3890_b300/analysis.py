"""Trajectory observables of pulled wires: yield stress and strain, failure
strain and final-neck atom count (Results, "Nanowire elongation"; Table 3
reports these per temperature and size without defining them).

Readings, taken on the reports of a run (per-wire observables and
tbsma_wire_topology every `report_every` steps):
  yield     sigma_y = the largest value of sigma_xx averaged over the reports
            of the last `window_fs` (0.5 ps by default; a trailing mean),
            eps_y = the strain at that report;
  failure   eps_f = the strain at the first report at which the two grips
            are no longer in one cluster of interacting atoms;
  neck      the neck count (fewest atoms in a (100)-plane slab between the
            grips) at the last report before failure;
  end       a run stops when every wire has failed and been pulled 2 A past
            its failure (Methods: the runs continue 2 A beyond failure), or
            after `max_steps`.
This module only reads what the library reports; it does no MD arithmetic.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np


def trailing_mean(y: np.ndarray, k: int) -> np.ndarray:
    """Mean of the last k values at every index (fewer at the start)."""
    y = np.asarray(y, dtype=np.float64)
    k = max(1, int(k))
    c = np.concatenate([[0.0], np.cumsum(y)])
    i = np.arange(1, y.size + 1)
    lo = np.maximum(0, i - k)
    return (c[i] - c[lo]) / (i - lo)


def yield_point(strain, sigma, window: int = 1) -> tuple[float, float]:
    """(sigma_y, eps_y): the maximum of the trailing mean of sigma over
    `window` reports and the strain at which it occurs (first on ties)."""
    s = trailing_mean(sigma, window)
    if s.size == 0:
        return math.nan, math.nan
    k = int(np.argmax(s))
    return float(s[k]), float(np.asarray(strain)[k])


def failure(strain, connected, neck) -> tuple[float, int]:
    """(eps_f, final neck): the strain of the first disconnected report and
    the neck count at the report before it (nan, -1 if the wire never fails;
    the neck of the first report if it fails at once)."""
    connected = np.asarray(connected, dtype=bool)
    off = np.flatnonzero(~connected)
    if off.size == 0:
        return math.nan, -1
    k = int(off[0])
    return float(np.asarray(strain)[k]), int(np.asarray(neck)[max(k - 1, 0)])


@dataclasses.dataclass
class WireResult:
    sigma_y: float  # eV/A^3
    eps_y: float
    eps_f: float  # nan if the wire did not fail
    final_neck: int  # -1 if it did not fail
    strain: np.ndarray
    sigma: np.ndarray
    connected: np.ndarray
    neck: np.ndarray


EV_PER_A3_IN_GPA = 160.21766208  # 1 eV/A^3 in GPa


def pull_to_rupture(eng, report_every: int, max_steps: int, dt: float = 2.0,
                    window_fs: float = 500.0, past_failure: float = 2.0) -> list[WireResult]:
    """Step an Engine in blocks of `report_every` steps, reporting observables
    and topology after each block, until every wire failed and was pulled
    `past_failure` A further (or `max_steps`); returns one WireResult per wire."""
    W = eng.W
    L0 = np.asarray(eng.batch.L0, dtype=np.float64)
    strain, sigma, conn, neck = [], [], [], []
    first_off = np.full(W, -1)
    done = 0
    while done + report_every <= max_steps:
        eng.step(report_every, dt)
        done += report_every
        ob = eng.observables()
        top = eng.topology()
        strain.append(ob["strain"].copy())
        sigma.append(ob["sigma_xx"].copy())
        conn.append(top["connected"].copy())
        neck.append(top["neck"].copy())
        k = len(strain) - 1
        first_off[(first_off < 0) & ~top["connected"]] = k
        if np.all(first_off >= 0):
            eps_f = np.array([strain[first_off[w]][w] for w in range(W)])
            if np.all((ob["strain"] - eps_f) * L0 >= past_failure):
                break
    strain, sigma = np.array(strain).reshape(-1, W), np.array(sigma).reshape(-1, W)
    conn, neck = np.array(conn).reshape(-1, W), np.array(neck).reshape(-1, W)
    window = max(1, int(round(window_fs / (report_every * dt))))
    out = []
    for w in range(W):
        sy, ey = yield_point(strain[:, w], sigma[:, w], window)
        ef, fn = failure(strain[:, w], conn[:, w], neck[:, w])
        out.append(WireResult(sy, ey, ef, fn, strain[:, w], sigma[:, w], conn[:, w], neck[:, w]))
    return out

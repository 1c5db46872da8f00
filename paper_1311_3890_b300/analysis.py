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
  mode      the post-yield strain eps_f - eps_y separates brittle failure
            (the wire fails right after yielding) from ductile failure; the
            paper shows the bimodal distributions (Figures 4-8) without a
            numeric cut, so the cut is a parameter (default 0.1);
  L_C       Eq. 6, L_C = (D0 / eps_y) cot(alpha) with cot(alpha) from 1
            (perfect dislocations) to sqrt(2) (partial dislocations) for
            [100] wires; the observed L_C is the midpoint between the
            longest L0 with predominantly ductile failure and the shortest
            L0 with predominantly brittle failure.
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


def critical_length(d0_nm: float, eps_y: float) -> tuple[float, float]:
    """Eq. 6 range (nm): (D0/eps_y) cot(alpha) for cot(alpha) = 1 and sqrt(2)."""
    base = d0_nm / eps_y
    return base, base * math.sqrt(2.0)


def post_yield_strain(eps_f, eps_y) -> np.ndarray:
    return np.asarray(eps_f, dtype=np.float64) - np.asarray(eps_y, dtype=np.float64)


def brittle(eps_f, eps_y, cut: float = 0.1) -> np.ndarray:
    """True where the wire failed within `cut` of strain after yielding."""
    return post_yield_strain(eps_f, eps_y) < cut


def observed_critical_length(lengths, eps_f, eps_y, cut: float = 0.1) -> float:
    """Midpoint between the longest initial length whose wires fail mostly
    (>= half) ductile and the shortest one whose wires fail mostly brittle,
    over groups of wires by initial length (nan if no such pair)."""
    lengths = np.asarray(lengths, dtype=np.float64)
    b = brittle(eps_f, eps_y, cut)
    groups = sorted(set(lengths.tolist()))
    frac = {L: float(np.mean(b[lengths == L])) for L in groups}
    ductile = [L for L in groups if frac[L] < 0.5]
    brit = [L for L in groups if frac[L] >= 0.5]
    if not ductile or not brit:
        return math.nan
    lo = max(L for L in ductile if L < min(brit)) if any(L < min(brit) for L in ductile) else None
    if lo is None:
        return math.nan
    return 0.5 * (lo + min(L for L in brit if L > lo))


def failure_map(lengths, eps_f, eps_y, length_edges, strain_edges) -> np.ndarray:
    """Counts of wires per (initial length, post-yield strain) bin: the
    histograms behind the paper's failure heat maps."""
    h, _, _ = np.histogram2d(np.asarray(lengths, dtype=np.float64),
                             post_yield_strain(eps_f, eps_y),
                             bins=[np.asarray(length_edges), np.asarray(strain_edges)])
    return h


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


@dataclasses.dataclass
class PaperRun:
    log_stretch: np.ndarray  # barostat lambda per wire after the equilibration
    results: list  # WireResult per wire, strains relative to the equilibrated length


def paper_protocol(eng, barostat_steps: int = 50000, ramp_steps: int = 200000,
                   hold_steps: int = 200000, pull_step: float = 0.05,
                   pull_interval: int = 10000, report_every: int = 1000,
                   max_pull_steps: int = 2_000_000, dt: float = 2.0, tau_fs: float = 1000.0,
                   baro_tau_fs: float = 1000.0, t_start: float = 0.01,
                   window_fs: float = 500.0) -> PaperRun:
    """The paper's protocol (Methods, "Simulation details") on every wire of
    an Engine, from its current state: (1) barostat_steps (100 ps) at zero
    axial pressure with the Nosé–Hoover barostat and a Nosé–Hoover target of
    t_start (0.01 K); (2) ramp_steps (400 ps) ramping the target from t_start
    to each wire's temperature; (3) hold_steps (400 ps) at that temperature;
    the grips do not move in (1)-(3).  Then the elongation: each grip moves
    by pull_step (0.05 A) every pull_interval steps (20 ps) until every wire
    has failed (pull_to_rupture).  The strains of the results are measured
    against the equilibrated length L0 e^lambda (the barostat's log-stretch),
    so a failure strain is the paper's elongation over the relaxed wire.
    Every phase sets the protocol anew, which restarts the thermostat
    variable; the steps keep counting from tbsma_init."""
    s0 = int(np.asarray(eng.observables()["step"])[0])
    common = dict(thermostat="nose_hoover", tau_fs=tau_fs, t_start=t_start,
                  ramp_steps=max(1, int(ramp_steps)), ramp_start=s0 + int(barostat_steps))
    hold = dict(pull="stepwise", pull_step=0.0, pull_interval=1)
    eng.set_protocol(**common, **hold, baro_tau_fs=baro_tau_fs)
    if barostat_steps > 0:
        eng.step(int(barostat_steps), dt)
    lam = np.asarray(eng.barostat()[0], dtype=np.float64).copy()
    eng.set_protocol(**common, **hold)
    if ramp_steps + hold_steps > 0:
        eng.step(int(ramp_steps + hold_steps), dt)
    eng.set_protocol(**common, pull="stepwise", pull_step=pull_step,
                     pull_interval=int(pull_interval))
    res = pull_to_rupture(eng, report_every=report_every, max_steps=max_pull_steps, dt=dt,
                          window_fs=window_fs)
    for r, lw in zip(res, lam):
        f = math.exp(-lw)  # strain = 2 d_grip / L0  ->  2 d_grip / (L0 e^lambda)
        r.strain = r.strain * f
        r.eps_y *= f
        r.eps_f *= f
    return PaperRun(lam, res)


@dataclasses.dataclass
class Campaign:
    lengths_nm: np.ndarray  # initial length per wire
    log_stretch: np.ndarray
    eps_y: np.ndarray
    sigma_y: np.ndarray  # eV/A^3
    eps_f: np.ndarray  # nan where a wire did not fail
    final_neck: np.ndarray
    brittle: np.ndarray  # post-yield strain below the cut
    critical_length_nm: float  # observed L_C (nan without a ductile/brittle pair)
    failure_map: np.ndarray  # counts per (length bin, post-yield strain bin)
    length_edges: np.ndarray
    strain_edges: np.ndarray


def campaign(eng, lengths_nm, length_edges=None, strain_edges=None, cut: float = 0.1,
             **protocol) -> Campaign:
    """The paper's statistical experiment on a batch (Results, "Nanowire
    elongation"; Figures 4-10, Eq. 6): the whole protocol on every wire of
    `eng` (paper_protocol, keyword arguments passed on), then per wire the
    yield point, failure strain and final neck, the brittle/ductile split at
    post-yield strain `cut`, the failure map over (initial length,
    post-yield strain) bins and the observed critical length.  `lengths_nm`
    gives each wire's initial length (the batch's own wire order)."""
    run = paper_protocol(eng, **protocol)
    L = np.asarray(lengths_nm, dtype=np.float64)
    eps_y = np.array([r.eps_y for r in run.results])
    eps_f = np.array([r.eps_f for r in run.results])
    if length_edges is None:
        u = np.unique(L)
        mids = 0.5 * (u[1:] + u[:-1]) if u.size > 1 else np.array([])
        length_edges = np.concatenate([[u[0] - 1.0], mids, [u[-1] + 1.0]])
    if strain_edges is None:
        strain_edges = np.linspace(0.0, 1.0, 21)
    ok = np.isfinite(eps_f)
    return Campaign(
        lengths_nm=L, log_stretch=run.log_stretch, eps_y=eps_y,
        sigma_y=np.array([r.sigma_y for r in run.results]), eps_f=eps_f,
        final_neck=np.array([r.final_neck for r in run.results]),
        brittle=np.where(ok, brittle(np.where(ok, eps_f, 0.0), eps_y, cut), False),
        critical_length_nm=observed_critical_length(L[ok], eps_f[ok], eps_y[ok], cut),
        failure_map=failure_map(L[ok], eps_f[ok], eps_y[ok], length_edges, strain_edges),
        length_edges=np.asarray(length_edges), strain_edges=np.asarray(strain_edges))


def save_results(path: str, results) -> None:
    """Per-wire report histories and readings of pull_to_rupture or
    paper_protocol into one compressed .npz (wire w's arrays under
    "w{w}_strain", "w{w}_sigma", "w{w}_connected", "w{w}_neck"; the readings
    as arrays over wires)."""
    arrays = {}
    for w, r in enumerate(results):
        arrays[f"w{w}_strain"] = np.asarray(r.strain)
        arrays[f"w{w}_sigma"] = np.asarray(r.sigma)
        arrays[f"w{w}_connected"] = np.asarray(r.connected)
        arrays[f"w{w}_neck"] = np.asarray(r.neck)
    for k in ("sigma_y", "eps_y", "eps_f", "final_neck"):
        arrays[k] = np.array([getattr(r, k) for r in results])
    np.savez_compressed(path, **arrays)

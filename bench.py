#!/usr/bin/env python
"""Aggregate TB-SMA atom-steps/s of the batched mixed-precision wire MD step.

Workload (default): the statistical sweep of 2048 independent Au [100]
wires, D in {2, 3, 4} nm x 24 lengths from 5 to 120 nm x T in {10, 298} K
(trajectory t takes class t mod 144), 55.8M atoms, Philox seeds 0..2047,
strain rate 1e8 1/s, dt = 2 fs, synthetic fcc geometry (the paper's >2000
trajectories of Results, "Nanowire elongation").  The wires start from the
perfect lattice with Gaussian velocities at T and run 2000 untimed
equilibration steps (surface relaxation and the thermostat bring the list
rebuild cadence to its steady state), then W warm-up steps, then K timed
steps.  One bench step = one MD step of every wire: B A O A, displacement
check, list rebuilds as they occur, density pass, force pass, B; the
per-wire observables are reduced after every 1000 timed steps and at the end.
Inputs (~25 GB of state and lists) are far larger than the 126 MB L2, so no
flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload NAME]

Under torchrun each rank runs its own full batch (seeds offset by rank):
weak scaling, no collective on the data path; rank 0 prints one JSON line.
`--impl reference` times the FP64 CPU oracle on a bounded sample of the same
workload on this host's cores (rank 0 only).
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "sweep2048"
EQUIL_STEPS = 2000  # untimed equilibration before the warm-up steps (steady rebuild cadence)
LAUNCH = (256, 1280)  # pair passes: atoms per tile (threads per block), shared-memory window (atoms)
GRAPH_CHUNK = 50  # steps per captured graph (library constant)
PERSIST_STEPS = 1000  # most steps per launch of the persistent step kernel (library constant)
# List skin (A).  Results do not depend on it (every pass tests r_cut); at
# 10 K a 0.40 A skin keeps the list radius (6.20 A) inside the gap between the
# fourth (5.77 A) and fifth (6.45 A) fcc shells, so the lists are no longer
# while rebuilds, driven by thermal excursions past skin/2, become ~15x rarer
# than at 0.29 A (measured on this workload: 751.6 -> 700.6 us per step).
R_SKIN = 0.40
KERNELS_PER_STEP = 4  # integrate, plan, density, force (+ the rebuild chain when it runs)
KERNELS_PER_CHAIN = 7  # two envelope passes, cell clear, bin, sort, cell build, slab build (per plan)
OBS_EVERY = 1000  # per-wire observables reported every OBS_EVERY steps inside the timed region
KERNELS_PER_OBS = 5  # pack, plan, density + force (with energies), reduce (+ a rebuild chain)
# a report folded into the call's last step (tbsma_step_observe in graph
# replays): that step's passes form the energies, so the report is the reduce
KERNELS_PER_FOLDED_OBS = 1
METRIC = "aggregate TB-SMA atom-steps/s (batched FP32/FP64-mixed vs plain FP64) at ≤1e-5 force err"
UNIT = "atom-steps/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10000)
    p.add_argument("--warmup", type=int, default=100, help="untimed steps after the equilibration")
    p.add_argument("--equil", type=int, default=EQUIL_STEPS,
                   help="untimed equilibration steps from the lattice start (part of the input "
                        "recipe: the rebuild cadence is then in steady state)")
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default=WORKLOAD)
    p.add_argument("--e2e-seg", type=int, default=100, help="MD steps per end-to-end segment")
    p.add_argument("--autotune", action="store_true",
                   help="pick the pair passes' launch shape with the autotuner first")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the cpu baseline, fp64 comparison and e2e legs")
    p.add_argument("--potential", default="tbsma", choices=["tbsma", "eam"],
                   help="eam: the tabulated-EAM pair passes (tbsma_set_eam) on Au tables that "
                        "sample the TB-SMA functions (every leg, the oracle's included)")
    p.add_argument("--table2", action="store_true",
                   help="context: steps/s of the paper's Table 2 wires, each alone, 10 and 298 K")
    p.add_argument("--precision", default="mixed", choices=["mixed", "fp64"],
                   help="arithmetic of the timed context (fp64: the plain FP64 path)")
    p.add_argument("--run-log", default=None,
                   help="time the run through runlog.run_logged into this JSON-lines file: "
                        "observables every 1000 steps and the mixed-vs-FP64 force check at each")
    p.add_argument("--r-skin", type=float, default=R_SKIN,
                   help="neighbour-list skin, A (forces do not depend on it)")
    p.add_argument("--lanes", type=int, default=1, choices=[1, 2, 4],
                   help="threads per atom in the pair passes (bitwise the same results)")
    p.add_argument("--step-mode", default="auto", choices=["auto", "graph", "persistent"],
                   help="graph replays or the persistent step kernel (auto: persistent where "
                        "the context can run it)")
    return p.parse_args()


def _env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


# --------------------------------------------------------------- clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def mark(self):
        """The timed region starts: samples taken before this are not reported."""
        try:
            with open(self.path) as f:
                self.skip = sum(1 for _ in f)
        except Exception:
            self.skip = 0

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)  # at least one sample after the timed region's start
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = open(self.path).readlines()
        keep = lines[getattr(self, "skip", 0):] or lines[-1:]
        for line in keep:
            parts = [t.strip() for t in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------- wire samples
def strata_of(specs):
    """Wires grouped by (diameter, temperature): {key: [wire indices]}."""
    out = {}
    for w, sp in enumerate(specs):
        out.setdefault((float(sp.diameter_nm), float(sp.temperature)), []).append(w)
    return dict(sorted(out.items()))


def stratified_sample(specs, atoms, per_stratum: int):
    """per_stratum wires of every (diameter, temperature) stratum, spread
    evenly over the stratum's sizes (atoms[w]); largest first."""
    picks = []
    for ws in strata_of(specs).values():
        order = sorted(ws, key=lambda w: (atoms[w], w))
        k = min(per_stratum, len(order))
        idx = sorted({int(round((j + 0.5) / k * len(order) - 0.5)) for j in range(k)})
        picks += [order[i] for i in idx]
    return sorted(picks, key=lambda w: (-atoms[w], w))


def extrapolate(specs, atoms, sampled: dict) -> float:
    """Workload rate from per-wire samples {w: (atom_steps, seconds)}: the
    rate of each (diameter, temperature) stratum is its samples' atom-steps
    over their time; the workload's time per step is the sum over strata of
    the stratum's atoms over its rate."""
    t = 0.0
    total = 0
    for ws in strata_of(specs).values():
        got = [sampled[w] for w in ws if w in sampled]
        rate = sum(a for a, _ in got) / sum(s for _, s in got)
        n = sum(int(atoms[w]) for w in ws)
        t += n / rate
        total += n
    return total / t


def _subbatch(batch, wires):
    """The wires `wires` of a batch (in that order) as a new batch."""
    from inputs.wires import Wire, pack

    out = []
    for w in wires:
        s = batch.wire_slice(w)
        out.append(Wire(x=batch.x[s].copy(), kind=batch.kind[s].copy(), diameter_nm=0.0,
                        length_nm=0.0, L0=float(batch.L0[w]),
                        temperature=float(batch.temperature[w]),
                        strain_rate=float(batch.strain_rate[w]), gamma=float(batch.gamma[w]),
                        seed=int(batch.seed[w])))
    return pack(out)


# --------------------------------------------------------- CPU oracle leg
def oracle_sample(batch, budget_s: float, steps: int | None = None, eam: bool = False,
                  wires=None):
    """Time the FP64 oracle on sample wires of the batch (default: the first
    wires), one wire per task over the host threads, largest first (eam:
    with the Au EAM tables of au_eam_tables in place of TB-SMA).

    Returns (atom-steps/s, threads used, description, atoms, steps)."""
    import oracle

    kw = {"pot": oracle.EamPotential(oracle.EamTables(**au_eam_tables(), r_cut=5.8))} if eam else {}

    threads = oracle.max_threads()
    if wires is None:
        wires = list(range(min(threads, batch.n_wires)))
    sub = _subbatch(batch, wires)
    W = sub.n_wires
    n = sub.n
    N = int(n.sum())
    x = sub.x.copy()
    v = np.zeros_like(x)
    args = (sub.kind, sub.offset, n, sub.L0, sub.strain_rate, sub.temperature, sub.gamma, sub.seed)
    F, xb, dg, nr = oracle.md_batch(x, v, *args, 0, 1, 2.0, brute_max=0, **kw)  # includes first forces
    t = time.perf_counter()
    oracle.md_batch(x, v, *args, 1, 1, 2.0, brute_max=0, F=F, x_build=xb, d_grip=dg, n_rebuild=nr,
                    **kw)
    per_step = time.perf_counter() - t
    if steps is None:
        steps = int(max(2, min(500, budget_s / max(per_step, 1e-6))))
    t = time.perf_counter()
    oracle.md_batch(x, v, *args, 2, steps, 2.0, brute_max=0, F=F, x_build=xb, d_grip=dg,
                    n_rebuild=nr, **kw)
    el = time.perf_counter() - t
    desc = (f"{W} of {batch.n_wires} wires ({N} atoms; one wire per task, {min(threads, W)} "
            f"host threads) x {steps} MD steps")
    if eam:
        desc += ", tabulated EAM"
    return N * steps / el, min(threads, W), desc, N, steps


def _oracle_run(batch, first_step: int, steps: int, state=None, eam: bool = False):
    """Run the FP64 oracle on a batch (one wire per host thread; eam: with the
    Au EAM tables of au_eam_tables); returns the state."""
    import oracle

    kw = {"pot": oracle.EamPotential(oracle.EamTables(**au_eam_tables(), r_cut=5.8))} if eam else {}

    N = int(batch.n.sum())
    W = len(batch.n)
    a = (batch.kind[:N], batch.offset[:W], batch.n, batch.L0[:W], batch.strain_rate[:W],
         batch.temperature[:W], batch.gamma[:W], batch.seed[:W])
    if state is None:
        x, v = batch.x[:N].copy(), np.zeros((N, 3))
        for w in range(W):  # Gaussian velocities at T, as the GPU arm starts
            s = slice(int(batch.offset[w]), int(batch.offset[w]) + int(batch.n[w]))
            v[s] = oracle.init_velocities(batch.kind[s], int(batch.seed[w]),
                                          float(batch.temperature[w]))
        F, xb, dg, nr = oracle.md_batch(x, v, *a, 0, 0, 2.0, brute_max=0, **kw)
        state = (x, v, F, xb, dg, nr)
    x, v, F, xb, dg, nr = state
    oracle.md_batch(x, v, *a, first_step, steps, 2.0, brute_max=0, F=F, x_build=xb, d_grip=dg,
                    n_rebuild=nr, **kw)
    return state


def _workload_atoms(specs) -> int:
    """Atoms of the whole workload (geometry only, cached per wire shape)."""
    from inputs.configs import _geometry

    return int(sum(_geometry(float(sp.diameter_nm), float(sp.length_nm)).n for sp in specs))


def _spec_atoms(specs):
    from inputs.configs import _geometry

    return [_geometry(float(sp.diameter_nm), float(sp.length_nm)).n for sp in specs]


def workload_config(specs) -> dict:
    """The workload's shape for the JSON line's config."""
    d = sorted({float(sp.diameter_nm) for sp in specs})
    L = sorted({float(sp.length_nm) for sp in specs})
    T = sorted({float(sp.temperature) for sp in specs})
    rates = sorted({float(sp.strain_rate) for sp in specs})
    return {"wires": len(specs), "diameters_nm": d,
            "lengths_nm": L if len(L) <= 4 else f"{len(L)} from {L[0]:g} to {L[-1]:g}",
            "temperatures_K": T, "strain_rate_per_s": rates[0] if len(rates) == 1 else rates}


def run_reference(args):
    """The oracle as it stands, timed on the host on a bounded sample of the workload."""
    rank, world, _ = _env_rank()
    if rank != 0:
        return 0
    import oracle
    from inputs.configs import WORKLOADS, WireSpec, build

    threads = oracle.max_threads()
    specs = WORKLOADS[args.workload]()
    atoms = _spec_atoms(specs)
    total = args.steps + args.warmup
    budget_s = 120.0
    eam = args.potential == "eam"
    # a stratified sample: three wires per host thread, spread over the
    # (diameter, temperature) strata and their sizes, largest first
    n_strata = len(strata_of(specs))
    picks = stratified_sample(specs, atoms, max(1, (3 * threads + n_strata - 1) // n_strata))
    sample_specs = [specs[w] for w in picks]
    # one step of the sample sizes it
    probe = build(sample_specs)
    st = _oracle_run(probe, 0, 1, eam=eam)
    t = time.perf_counter()
    _oracle_run(probe, 1, 1, st, eam=eam)
    t_step = time.perf_counter() - t
    if total * t_step <= budget_s:
        sample = (f"{len(sample_specs)} of {len(specs)} wires of the workload, whole, stratified over "
                  f"diameter and temperature, one wire per task on {threads} host threads")
    else:
        # the same wires shortened (same diameter, temperature, pull and seeds) so
        # that warm-up + timed steps fit the budget: per-atom work of the oracle
        # is that of the full wires (same cross-section and neighbourhoods)
        frac = budget_s / (total * t_step)
        sample_specs = [WireSpec(sp.diameter_nm, max(3.0, round(sp.length_nm * frac, 1)),
                                 sp.temperature, sp.strain_rate, sp.seed, sp.gamma)
                        for sp in sample_specs]
        sample = (f"{len(sample_specs)} of {len(specs)} wires of the workload, stratified over "
                  f"diameter and temperature, each shortened to {100 * frac:.1f} % of its length "
                  f"(at least 3 nm) so that {total} steps fit ~{budget_s:.0f} s, one wire per "
                  f"task on {threads} host threads")
    sub = build(sample_specs)
    N = int(sub.n.sum())
    st = _oracle_run(sub, 0, max(1, args.warmup), eam=eam)
    t = time.perf_counter()
    _oracle_run(sub, max(1, args.warmup), args.steps, st, eam=eam)
    el = time.perf_counter() - t
    value = N * args.steps / el
    cfg = {"workload": args.workload, "atoms_per_gpu": _workload_atoms(specs), "dt_fs": 2.0}
    cfg.update(workload_config(specs))
    cfg.update({"precision": "fp64 (oracle)", "observables_every": None,
                "potential": "tabulated EAM (TB-SMA sampled)" if eam else "TB-SMA (Eq. 1-3)",
                "l2": "host", "parallelism": f"{threads} host threads"})
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": cfg,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads,
                         "kind": "oracle", "sample": f"{sample}; {N} atoms"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------- our path
def _chunks(K: int):
    """The timed call sequence: K steps in blocks of OBS_EVERY, observables after each."""
    out = []
    while K > 0:
        out.append(min(OBS_EVERY, K))
        K -= out[-1]
    return out


def launches_in(K: int, chains: int, persistent: bool = False) -> int:
    """Kernels launched by K timed steps in calls of tbsma_step_observe: the
    fixed ones per step, one closing kernel per graph replay or direct
    sequence, the report's reduce (folded into the call's last step), and
    `chains` launches of the rebuild chain (counted on the device).  In the
    persistent step kernel a call of up to 1000 steps is one launch, and the
    report runs its own passes: only the reports launch the rebuild chain."""
    if persistent:
        return sum(-(-k // PERSIST_STEPS) + KERNELS_PER_OBS + KERNELS_PER_CHAIN
                   for k in _chunks(K))
    n = KERNELS_PER_CHAIN * chains
    for k in _chunks(K):
        full, rem = divmod(k, GRAPH_CHUNK) if k >= GRAPH_CHUNK else (0, k)
        n += full * (KERNELS_PER_STEP * GRAPH_CHUNK + 1)
        if rem:
            n += KERNELS_PER_STEP * rem + 1
        n += KERNELS_PER_FOLDED_OBS
    return n


# Algorithmic work of the pair passes per in-cutoff pair (list entry with
# r <= r_cut; n_c per atom, both sides of each pair counted): the method's
# arithmetic, without list decoding, addressing or the fixed-point
# conversions of this implementation.
#   force pass  19 FP32: 3 coordinate differences, r^2 (3), the cutoff test,
#               r = r^2 rsqrt(r^2) (1), s (1), two exponent arguments (2), the
#               bracket (a_i + a_j, fp h minus that, times g: 3), f/r (1), the
#               three force components (3), one Newton step on r (1);
#               3 MUFU (rsqrt, two ex2)
#   density     11 FP32: differences (3), r^2 (3), test (1), r (1), the
#               exponent argument (1), the term (1), the sum (1); 2 MUFU
# HBM bytes per atom of one launch (the list stays in HBM): 2 per list
# entry (int16; skin entries included) + 4 (count) + 8 (index range)
# + 16 (own packed position) + 12 (F, force pass) or 4 (a_i, density pass).
# Peaks: 128 FP32 lanes and 32 MUFU results per clock per SM (an ex2
# throughput measurement on this GPU gave 29.8/clk/SM), at the median SM
# clock sampled during the timed region; HBM from MEASURED_PEAKS.  The
# roofline time is the slower of the ALU time (FP32 and MUFU pipes run
# concurrently: the larger of the two) and the HBM time.
PASS_MODEL = {
    "force": {"fp32_in": 19, "fp32_skin": 0, "mufu_in": 3, "bytes_out": 12},
    "density": {"fp32_in": 11, "fp32_skin": 0, "mufu_in": 2, "bytes_out": 4},
}
# The force pass's instruction count in this implementation (the three
# int->float conversions per entry included, 7 per skin entry: conversions,
# r^2, test), reported beside the method's count.
FORCE_IMPL_MODEL = {"fp32_in": 21, "fp32_skin": 7, "mufu_in": 3, "bytes_out": 12}
# The tabulated-EAM force pass (--potential eam) per in-cutoff entry: the
# same geometry (6), radius (4, one MUFU rsqrt), bracket (2), scale (1) and
# accumulation (3), plus the interval and t of r (5: FMUL, F2I, I2F, two
# FFMA) and two quadratic derivative polynomials (4) in place of the two ex2;
# MUFU 1; skin entries as above.
EAM_MODEL = {"fp32_in": 25, "fp32_skin": 7, "mufu_in": 1, "bytes_out": 12}
# DRAM bytes (read + write) per atom of one force-pass launch from an ncu
# capture of the current kernel on a smaller case of the same workload
# (sweep144: 528.30 MB read + 41.71 MB written for 3,971,388 atoms), scaled
# by the atom count (the traffic is per atom); None once the kernel changes.
FORCE_TRAFFIC_B_PER_ATOM = 143.5


def au_eam_tables(d_r=0.002, d_rho=0.005, rho_max=120.0, r_cut=5.8):
    """Au as a tabulated EAM for the --potential eam line: the TB-SMA
    functions of Table 1 sampled on uniform grids (f = xi^2 e^{-2q s},
    phi = 2 A e^{-p s}, F = -sqrt(rho)), so that the EAM run has the TB-SMA
    run's dynamics and rebuild cadence and only the pair arithmetic differs."""
    A, xi, p, q, r0 = 0.2061, 1.790, 10.229, 4.036, 2.884
    r = np.arange(int(np.ceil((r_cut + 0.05) / d_r)) + 1) * d_r
    s = r / r0 - 1.0
    rho = np.arange(int(np.ceil(rho_max / d_rho)) + 1) * d_rho
    return dict(F=-np.sqrt(rho), d_rho=d_rho, f=xi * xi * np.exp(-2.0 * q * s),
                phi=2.0 * A * np.exp(-p * s), d_r=d_r)


def _list_census(eng, r_cut=5.8, chunk=1 << 20):
    """Mean in-cutoff and skin entries per atom of the current lists (on the GPU)."""
    import torch

    n, nb = eng.neighbors()
    N = eng.N
    x = eng.x.view(3, N)
    n_in = 0
    for s in range(0, N, chunk):
        rows = nb[s:s + chunk].long()
        valid = rows >= 0
        j = rows.clamp(min=0)
        d2 = torch.zeros(rows.shape, dtype=torch.float64, device=rows.device)
        for d in range(3):
            d2 += (x[d][j] - x[d][s:s + chunk, None]) ** 2
        n_in += int(((d2 <= r_cut * r_cut) & valid).sum().item())
    n_all = int(n.long().sum().item())
    return n_in / N, (n_all - n_in) / N


def roofline_of(N, n_c, n_s, ms, sms, mhz, hbm_gbs, model=PASS_MODEL["force"]):
    """A pair pass's roofline from its algorithmic work (per atom: n_c
    in-cutoff and n_s skin list entries, `model` the counts per entry) and
    its measured time per launch `ms`, for `sms` SMs at `mhz` and an HBM
    peak of `hbm_gbs`: the bound is the slower of the FP32 and MUFU pipes
    (which run concurrently) and the bytes at HBM bandwidth; `achieved` is
    the bound's work over the time."""
    f = mhz * 1e6
    fp32_ops = N * (model["fp32_in"] * n_c + model["fp32_skin"] * n_s)
    mufu_ops = N * model["mufu_in"] * n_c
    bytes_ = N * (2.0 * (n_c + n_s) + 4 + 8 + 16 + model["bytes_out"])
    t_fp32 = fp32_ops / (128 * sms * f)
    t_mufu = mufu_ops / (32 * sms * f)
    t_hbm = bytes_ / (hbm_gbs * 1e9)
    t = ms * 1e-3
    if max(t_fp32, t_mufu) >= t_hbm:
        if t_fp32 >= t_mufu:
            bound = {"bound": "alu", "achieved": fp32_ops / t / 1e12,
                     "peak": 128 * sms * f / 1e12, "unit": "T FP32-inst/s"}
        else:
            bound = {"bound": "alu", "achieved": mufu_ops / t / 1e12,
                     "peak": 32 * sms * f / 1e12, "unit": "T MUFU-op/s"}
    else:
        bound = {"bound": "hbm", "achieved": bytes_ / t / 1e9, "peak": hbm_gbs, "unit": "GB/s"}
    bound["frac"] = bound["achieved"] / bound["peak"]
    bound.update({
        "ms_per_launch": ms,
        "roofline_ms": 1e3 * max(t_fp32, t_mufu, t_hbm),
        "t_fp32_ms": 1e3 * t_fp32, "t_mufu_ms": 1e3 * t_mufu, "t_hbm_ms": 1e3 * t_hbm,
        "hbm_frac": bytes_ / t / 1e9 / hbm_gbs,
        "entries_in_cutoff": n_c, "entries_skin": n_s, "sm_mhz": mhz,
    })
    return bound


def pass_rooflines(eng, ms_force, ms_density, clocks, eam=False, captured=True):
    """The force pass's roofline (the dominant kernel), with the density
    pass's beside it.  `captured`: the force kernel runs in the launch shape
    and lane count its DRAM traffic was captured with."""
    import torch

    n_c, n_s = _list_census(eng)
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    hbm, kind = _peaks()
    sms, mhz = props.multi_processor_count, clocks.get("sm_mhz") or 2032.0
    force_model = EAM_MODEL if eam else PASS_MODEL["force"]
    bound = roofline_of(eng.N, n_c, n_s, ms_force, sms, mhz, hbm, model=force_model)
    traffic = (None if (eam or not captured or FORCE_TRAFFIC_B_PER_ATOM is None)
               else FORCE_TRAFFIC_B_PER_ATOM * eng.N)
    bound.update({
        "kernel": "k_force_f32<EAM>" if eam else "k_force_f32",
        "model": ("EAM: 25 FP32 + 1 MUFU per in-cutoff entry, 7 FP32 per skin entry" if eam else
                  "19 FP32 + 3 MUFU per in-cutoff pair (the method's arithmetic)"),
        "traffic": traffic,
        "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum per atom, small-case "
                          "capture of the same workload scaled by atoms",
        "hbm_peak_kind": kind,
    })
    if not eam:
        impl = roofline_of(eng.N, n_c, n_s, ms_force, sms, mhz, hbm, model=FORCE_IMPL_MODEL)
        bound["frac_impl_count"] = impl["frac"]
        d = roofline_of(eng.N, n_c, n_s, ms_density, sms, mhz, hbm, model=PASS_MODEL["density"])
        bound["density"] = {k: d[k] for k in ("bound", "achieved", "peak", "unit", "frac",
                                              "ms_per_launch", "roofline_ms")}
    else:
        bound["density_ms_per_launch"] = ms_density
    return bound


def fp64_one_wire_per_launch(tb, specs, batch, params, eam=False, steps=20):
    """The plain FP64 path, one wire per context, on a stratified sample of
    the workload's wires (two per diameter and temperature), extrapolated to
    the workload per stratum (see extrapolate)."""
    import torch

    picks = stratified_sample(specs, batch.n, 2)
    sampled = {}
    for w in picks:
        one = _subbatch(batch, [w])
        e1 = tb.Engine(one, precision="fp64", params=params)
        if eam:
            e1.set_eam(**au_eam_tables())
        e1.set_launch(64, 0)  # one wire: small tiles to spread it over the SMs
        e1.init_velocities()
        e1.step(5, 2.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        e1.step(steps, 2.0)
        b.record()
        torch.cuda.synchronize()
        sampled[w] = (one.n_atoms * steps, a.elapsed_time(b) / 1e3)
        e1.close()
    return {"value": extrapolate(specs, batch.n, sampled), "unit": UNIT,
            "sample": (f"{len(picks)} of {len(specs)} wires (two per diameter and temperature, "
                       f"spread over lengths), each alone in its own FP64 context, {steps} steps; "
                       f"per-stratum rates weighted by the workload's atoms")}


def run_ours(args):
    import torch
    import torch.distributed as dist

    from inputs.configs import WORKLOADS, build
    import paper_1311_3890_b300 as tb
    from paper_1311_3890_b300.shard import aggregate, replicate_specs

    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    specs = replicate_specs(WORKLOADS[args.workload](), rank, world)
    batch = build(specs)
    N, W = batch.n_atoms, batch.n_wires
    params = tb.au_params(r_skin=args.r_skin)
    eng = tb.Engine(batch, precision=args.precision, params=params)
    eam = args.potential == "eam"
    if eam:
        eng.set_eam(**au_eam_tables())
    launch = LAUNCH
    eng.set_launch(*launch)
    eng.set_pair_lanes(args.lanes)
    persist_blocks = eng.set_step_mode(args.step_mode)
    eng.init_velocities()
    # the input recipe: equilibrate from the lattice start (untimed), so that
    # surface relaxation is over and list rebuilds come at their steady rate
    if args.equil > 0:
        eng.step(args.equil, 2.0)
    if args.autotune:
        from paper_1311_3890_b300.autotune import tune

        launch, _ = tune(eng)
        eng.set_launch(*launch)
    # the clock sampler starts before the last warm-up steps, so that the GPU
    # does not idle (and drop its clocks) between them and the timed region
    clocks = Clocks(local)
    clocks.start()
    eng.step(max(3, args.warmup), 2.0)
    # one report outside the timed region too, so that the first use of its
    # kernels (module loading on first launch) is not timed
    eng.observables()
    # capture the step graph the timed calls will replay (50-step chunks, or
    # all K steps when K < 50) outside the timed region
    eng.step(min(_chunks(args.steps)[0], GRAPH_CHUNK), 2.0)
    rs0 = eng.rebuild_stats()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.mark()
    log = None
    if args.run_log:
        from paper_1311_3890_b300.runlog import RunLog, run_logged

        log = RunLog(args.run_log, workload=args.workload, precision=args.precision)
    ev0.record()
    if log is not None:  # the job through the run logger: reports and force checks every 1000
        # a report every 1000 steps, and the force check at every report
        ob = run_logged(eng, args.steps, log, 2.0, report_every=OBS_EVERY, check_every=1)
    else:
        for k in _chunks(args.steps):  # the job: steps with per-wire observables every OBS_EVERY
            ob = eng.step_observe(k, 2.0)
    ev1.record()
    torch.cuda.synchronize()
    ck = clocks.stop()
    if world > 1:
        dist.barrier()
    t_ms = ev0.elapsed_time(ev1)
    rs1 = eng.rebuild_stats()
    chains = rs1["chains"] - rs0["chains"]
    t_max, atoms_all = aggregate(t_ms, N, device="cuda")
    value = atoms_all * args.steps / (t_max / 1e3)

    # where the time goes: the next K steps enqueued directly with an event
    # after each phase (same kernels), then one observables report alone
    split_steps = min(args.steps, 500)
    ph = eng.step_profile(split_steps, 2.0)
    rs2 = eng.rebuild_stats()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    eng.observables()
    b.record()
    torch.cuda.synchronize()
    obs_ms = a.elapsed_time(b)

    # force-error gate on the final state (same positions, same list)
    fc = eng.force_check()

    # the pair passes timed alone with CUDA events on the library's stream
    reps = 20
    res = {}
    for which in (1, 2):
        eng.run_pass(which, 3)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        eng.run_pass(which, reps)
        b.record()
        torch.cuda.synchronize()
        res[which] = a.elapsed_time(b) / reps
    captured = (tuple(launch) == LAUNCH and args.lanes == 1 and args.r_skin == R_SKIN
                and args.workload in ("sweep2048", "sweep144"))
    roof = (pass_rooflines(eng, res[2], res[1], ck, eam=eam, captured=captured)
            if args.precision == "mixed" else None)
    cfg = {"workload": args.workload, "atoms_per_gpu": N, "dt_fs": 2.0}
    cfg.update(workload_config(specs))
    cfg.update({"precision": args.precision,
                "step_mode": ("persistent step kernel (%d blocks)" % persist_blocks
                              if persist_blocks else "graph replays of 50 steps"),
                "potential": "tabulated EAM (TB-SMA sampled)" if eam else "TB-SMA (Eq. 1-3)",
                "equilibration_steps": args.equil, "observables_every": OBS_EVERY,
                "r_skin_A": args.r_skin, "tile_atoms": launch[0], "window_atoms": launch[1],
                "pair_lanes": args.lanes,
                "launch": "autotuned" if args.autotune else "fixed",
                "l2": "inputs larger than L2 (no flush)", "parallelism": f"wires x{world}"})
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "mixed f32 pair / f64 state" if args.precision == "mixed" else "f64",
        "data": "synthetic", "config": cfg,
        "roofline": roof,
        "clocks": ck,
        "gpu_launches": launches_in(args.steps, chains, persistent=persist_blocks > 0),
        "force_check": {"max_err_scaled": float(fc["max_err_scaled"].max()),
                        "norm_err": float(fc["norm_err"].max()),
                        "max_err_raw": float(fc["max_err_raw"].max())},
        "timed_window": {
            "rebuilt_wires": rs1["wires"] - rs0["wires"],
            "rebuilt_atoms": rs1["atoms"] - rs0["atoms"],
            "rebuilt_atoms_per_atom_step": (rs1["atoms"] - rs0["atoms"]) / (N * args.steps),
            "reports": len(_chunks(args.steps)),
        },
        "run_log": None,
        "split": {
            "steps": split_steps,
            "how": "the steps after the timed window, enqueued directly with a CUDA event after "
                   "each phase (same kernels as the graph), then one observables report alone",
            "ms_per_step": {k: v / split_steps for k, v in ph.items()},
            "sum_ms_per_step": sum(ph.values()) / split_steps,
            "observables_ms_per_report": obs_ms,
            "rebuilt_wires": rs2["wires"] - rs1["wires"],
            "rebuilt_atoms": rs2["atoms"] - rs1["atoms"],
        },
    }

    if log is not None:
        from paper_1311_3890_b300.runlog import read_log

        log.close()
        recs = [r for r in read_log(args.run_log) if r["kind"] == "force_check"]
        line["run_log"] = {
            "path": args.run_log, "force_checks": len(recs),
            "max_err_scaled": max((max(r["max_err_scaled"]) for r in recs), default=None),
            "norm_err": max((max(r["norm_err"]) for r in recs), default=None)}

    if not args.no_extras and rank == 0:
        # end to end through the public API: pinned host state in, K steps in
        # segments, per-wire observables and state out every segment
        seg = max(1, min(args.e2e_seg, args.steps))
        n_seg = max(1, min(10, args.steps // seg))
        xh = torch.empty(3 * N, dtype=torch.float64).pin_memory()
        vh = torch.empty(3 * N, dtype=torch.float64).pin_memory()
        eng.download(xh, vh)
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(n_seg):
            eng.upload(xh, vh)
            eng.step_observe(seg, 2.0)
            eng.download(xh, vh)
        el = time.perf_counter() - t
        obs_bytes = W * 64
        line["e2e"] = {"value": N * seg * n_seg / el, "unit": UNIT,
                       "h2d_bytes_per_step": 48.0 * N / seg,
                       "d2h_bytes_per_step": (48.0 * N + obs_bytes) / seg,
                       "segment_steps": seg, "segments": n_seg}
        line["fp64_one_wire_per_launch"] = fp64_one_wire_per_launch(tb, specs, batch, params, eam)
        if world == 1:
            import oracle

            threads = oracle.max_threads()
            n_strata = len(strata_of(specs))
            picks = stratified_sample(specs, batch.n,
                                      max(1, (3 * threads + n_strata - 1) // n_strata))
            v, cores, desc, _, _ = oracle_sample(batch, budget_s=15.0, eam=eam, wires=picks)
            # one core: the sample's median-sized wire alone (one wire is one task)
            mid = sorted(picks, key=lambda w: batch.n[w])[len(picks) // 2]
            v1, _, desc1, _, _ = oracle_sample(batch, budget_s=2.0, eam=eam, wires=[mid])
            line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                    "sample": desc + ", stratified over diameter and temperature",
                                    "single_core": {"value": v1, "unit": UNIT, "sample": desc1}}
    eng.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


# The paper's Table 2: timesteps per second of one unstretched D3.1 nm wire
# per GPU (GTX 680, HOOMD-Blue + TB-SMA in FP32) at 10 K and 298 K.
TABLE2_ATOMS = [8823, 17673, 26523, 35373, 44223, 53073, 61923, 70773, 79623, 88473, 97323, 106173]
TABLE2_10K = [2536, 1723, 1311, 1045, 881, 758, 655, 584, 514, 470, 427, 396]
TABLE2_298K = [2286, 1507, 1141, 897, 717, 616, 550, 484, 409, 354, 330, 300]


def run_table2(args):
    """Each Table 2 wire alone in its own mixed-precision context (as the
    paper ran one system per GPU), in the default step mode (the persistent
    step kernel where the wire's tiles fit the GPU at once, which all twelve
    do), the library default list skin: steps/s over the timed steps after
    the warm-up, at 10 K and at 298 K.  Context only, one JSON line."""
    import torch

    from inputs.configs import WireSpec, build
    import paper_1311_3890_b300 as tb

    torch.cuda.set_device(0)
    steps, warm = min(args.steps, 1000), min(args.warmup, 500)
    rows = []
    for k in range(1, 13):
        row = {"k": k, "length_nm": round(20.4 * k, 1)}
        for T in (10.0, 298.0):
            batch = build([WireSpec(3.1, 20.4 * k, T, 0.0, k)])
            eng = tb.Engine(batch, precision="mixed")
            row[f"persistent_blocks_{int(T)}K"] = eng.set_step_mode("auto")
            eng.init_velocities()
            eng.step(warm, 2.0)
            eng.step(min(50, steps), 2.0)  # capture the graph outside the timed region
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            eng.step(steps, 2.0)
            b.record()
            torch.cuda.synchronize()
            row["atoms"] = int(batch.n_atoms)
            row[f"steps_per_s_{int(T)}K"] = steps / (a.elapsed_time(b) / 1e3)
            eng.close()
        row["paper_atoms"] = TABLE2_ATOMS[k - 1]
        row["paper_steps_per_s_10K"] = TABLE2_10K[k - 1]
        row["paper_steps_per_s_298K"] = TABLE2_298K[k - 1]
        rows.append(row)
    print(json.dumps({"context": "paper Table 2 systems, each wire alone per context (mixed "
                      "precision, B300) against the paper's GTX 680 FP32 steps/s",
                      "steps": steps, "warmup": warm, "rows": rows}))


def main():
    args = parse()
    if args.table2:
        return run_table2(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

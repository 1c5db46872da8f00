"""Workload definitions: synthetic Au [100] wires shaped like the paper's.

Each workload is a list of WireSpec (diameter, length, temperature, strain
rate, Philox seed).  The paper's own systems are D0 = 3.1-6.0 nm, L0 = 20-140
nm wires at 10-298 K (Methods, "Simulation details"); the workloads below use
diameters 2-4 nm and lengths 5-120 nm in the same regime.  Geometry is built
by `wires.fcc_wire`; nothing here computes the method.
"""

from __future__ import annotations

import dataclasses
import functools

import numpy as np

from .wires import Batch, Wire, fcc_wire, pack


@dataclasses.dataclass(frozen=True)
class WireSpec:
    diameter_nm: float
    length_nm: float
    temperature: float
    strain_rate: float
    seed: int
    gamma: float = 1.0e-3  # 1/fs (1 ps^-1)


@functools.lru_cache(maxsize=256)
def _geometry(diameter_nm: float, length_nm: float) -> Wire:
    return fcc_wire(diameter_nm, length_nm)


def build(specs: list[WireSpec]) -> Batch:
    wires = []
    for s in specs:
        g = _geometry(float(s.diameter_nm), float(s.length_nm))
        wires.append(
            Wire(
                x=g.x,
                kind=g.kind,
                diameter_nm=g.diameter_nm,
                length_nm=g.length_nm,
                L0=g.L0,
                temperature=s.temperature,
                strain_rate=s.strain_rate,
                gamma=s.gamma,
                seed=s.seed,
            )
        )
    return pack(wires)


def _single_d2_l6() -> list[WireSpec]:
    return [WireSpec(2.0, 6.0, 10.0, 1.0e9, 0)]


def _single_d3_l40() -> list[WireSpec]:
    return [WireSpec(3.0, 40.0, 10.0, 1.0e8, 0)]


def _batch256_d3_l40() -> list[WireSpec]:
    return [WireSpec(3.0, 40.0, 10.0, 1.0e8, s) for s in range(256)]


def _batch32_d3_l40() -> list[WireSpec]:
    return [WireSpec(3.0, 40.0, 10.0, 1.0e8, s) for s in range(32)]


def _ragged512() -> list[WireSpec]:
    rng = np.random.default_rng(0xC4)
    d = rng.choice([2.0, 3.0, 4.0], size=512)
    # lengths drawn on a 1 nm grid from [10, 60] nm so that geometries repeat
    length = rng.integers(10, 61, size=512).astype(np.float64)
    t = rng.choice([10.0, 298.0], size=512)
    return [
        WireSpec(float(d[w]), float(length[w]), float(t[w]), 1.0e8, w) for w in range(512)
    ]


def _sweep2048() -> list[WireSpec]:
    diam = [2.0, 3.0, 4.0]
    lengths = np.linspace(5.0, 120.0, 24)
    temps = [10.0, 298.0]
    classes = [(d, float(L), T) for d in diam for L in lengths for T in temps]
    out = []
    for t in range(2048):
        d, L, T = classes[t % len(classes)]
        out.append(WireSpec(d, L, T, 1.0e8, t))
    return out


def _sweep144() -> list[WireSpec]:
    """The first 144 trajectories of the sweep: one wire of every (D, L, T)
    class (3.9M atoms), the small case of the sweep's kernel shapes."""
    return _sweep2048()[:144]


def _paper_table2() -> list[WireSpec]:
    """The paper's benchmark systems (Table 2, Results "TB-SMA benchmarks"):
    unstretched D 3.1 nm wires of length 20.4 k nm, k = 1..12 (8.9k-106k
    atoms here against the paper's 8.8k-106k), 10 K, no pull."""
    return [WireSpec(3.1, 20.4 * k, 10.0, 0.0, k) for k in range(1, 13)]


def _tiny_batch() -> list[WireSpec]:
    """Three small wires of uneven size and temperature (parity tests)."""
    return [
        WireSpec(2.0, 6.0, 10.0, 1.0e9, 0),
        WireSpec(2.0, 3.5, 298.0, 1.0e9, 7),
        WireSpec(3.0, 4.0, 10.0, 1.0e9, 11),
    ]


WORKLOADS = {
    # one D2 nm x L6 nm wire (1035 atoms), 10 K, 1e9 1/s, FP64
    "wire_d2_l6": _single_d2_l6,
    # one D3 nm x L40 nm wire (17435 atoms), 10 K, 1e8 1/s, mixed vs FP64
    "wire_d3_l40": _single_d3_l40,
    # 256 D3 x L40 wires (4.46M atoms), seeds 0..255, 10 K, 1e8 1/s, mixed
    "batch256_d3_l40": _batch256_d3_l40,
    # 32 D3 x L40 wires (558k atoms): a smaller case of the same kernel shapes
    "batch32_d3_l40": _batch32_d3_l40,
    # 512 wires, D in {2,3,4} nm, L in [10,60] nm, T in {10,298} K, mixed
    "ragged512": _ragged512,
    # 2048 trajectories over D {2,3,4} x 24 lengths 5..120 nm x T {10,298}
    "sweep2048": _sweep2048,
    # one wire of each of the sweep's 144 classes (3.9M atoms): its small case
    "sweep144": _sweep144,
    # the paper's Table 2 systems: D3.1 x L20.4k nm, k = 1..12, 10 K, no pull
    "paper_table2": _paper_table2,
    "tiny_batch": _tiny_batch,
}


def workload(name: str) -> Batch:
    return build(WORKLOADS[name]())

"""fcc Au [100] nanowire geometry (Methods, "Simulation details").

A wire is the set of fcc sites a*(n + b), n integer, b one of the four fcc
basis vectors, with the wire axis along [100] = x through an atom column at
y = z = 0.  Sites with y^2 + z^2 <= (D/2)^2 and 0 <= x < L are kept.  The two
lowest and the two highest x planes (planes are a/2 apart) are the rigid
"gripping" layers of Fig. 1.  Atoms are ordered along the [100] axis, the
ordering the paper found fastest on its GPU code (Results, "TB-SMA
benchmarks").

Everything here is input generation: lattice sites, labels and packing.
"""

from __future__ import annotations

import dataclasses

import numpy as np

# Lattice parameter of Au (Table 1 prints 4.079 in the r0 column; it is the
# fcc lattice constant, the nearest-neighbour distance being 4.079/sqrt(2)).
A_LATTICE = 4.079

KIND_MOBILE = 0
KIND_GRIP_LEFT = 1
KIND_GRIP_RIGHT = 2

_FCC_BASIS = np.array(
    [[0.0, 0.0, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]]
)


@dataclasses.dataclass
class Wire:
    """One wire: positions (n, 3) in Angstrom, kind (n,) uint8, and metadata."""

    x: np.ndarray
    kind: np.ndarray
    diameter_nm: float
    length_nm: float
    L0: float  # initial length = distance between the outermost x planes (Angstrom)
    temperature: float = 10.0  # K
    strain_rate: float = 0.0  # 1/s
    gamma: float = 1.0e-3  # Langevin friction, 1/fs
    seed: int = 0

    @property
    def n(self) -> int:
        return int(self.x.shape[0])


def _order_along_axis(x: np.ndarray) -> np.ndarray:
    """Permutation sorting atoms by (x, y, z), coordinates rounded to 1e-6 A."""
    r = np.round(x, 6)
    return np.lexsort((r[:, 2], r[:, 1], r[:, 0]))


def fcc_wire(
    diameter_nm: float,
    length_nm: float,
    a: float = A_LATTICE,
    grip_planes: int = 2,
    temperature: float = 10.0,
    strain_rate: float = 0.0,
    gamma: float = 1.0e-3,
    seed: int = 0,
    notch_depth: float = 0.0,
    notch_planes: int = 2,
) -> Wire:
    """Cylindrical [100] fcc wire of diameter D and length L (nm).

    notch_depth > 0 cuts a ring-shaped notch at the centre (Methods,
    "Simulation details": a small ring notch fixes where the wire breaks; its
    size is not given): the atoms farther than R_max - notch_depth from the
    axis are removed from the `notch_planes` (100) planes nearest the middle,
    R_max the largest radius of the wire's atoms."""
    R = 5.0 * diameter_nm  # radius in Angstrom
    L = 10.0 * length_nm
    nx = int(np.ceil(L / a)) + 1
    ny = int(np.ceil(R / a)) + 1
    i = np.arange(nx)
    j = np.arange(-ny, ny + 1)
    n = np.stack(np.meshgrid(i, j, j, indexing="ij"), axis=-1).reshape(-1, 1, 3)
    sites = (a * (n + _FCC_BASIS[None, :, :])).reshape(-1, 3)
    keep = (
        (sites[:, 1] ** 2 + sites[:, 2] ** 2 <= R * R + 1e-9)
        & (sites[:, 0] >= -1e-9)
        & (sites[:, 0] < L - 1e-9)
    )
    x = sites[keep]
    x = x[_order_along_axis(x)]
    planes = np.unique(np.round(x[:, 0], 6))
    if notch_depth > 0.0 and notch_planes > 0:
        mid = 0.5 * (planes[0] + planes[-1])
        centre = planes[np.argsort(np.abs(planes - mid), kind="stable")[:notch_planes]]
        r = np.hypot(x[:, 1], x[:, 2])
        cut = np.isin(np.round(x[:, 0], 6), centre) & (r > r.max() - notch_depth)
        x = x[~cut]
    kind = np.zeros(x.shape[0], dtype=np.uint8)
    if grip_planes > 0:
        lo = planes[grip_planes - 1]
        hi = planes[-grip_planes]
        kind[np.round(x[:, 0], 6) <= lo] = KIND_GRIP_LEFT
        kind[np.round(x[:, 0], 6) >= hi] = KIND_GRIP_RIGHT
    L0 = float(planes[-1] - planes[0])
    return Wire(
        x=np.ascontiguousarray(x),
        kind=kind,
        diameter_nm=float(diameter_nm),
        length_nm=float(length_nm),
        L0=L0,
        temperature=temperature,
        strain_rate=strain_rate,
        gamma=gamma,
        seed=seed,
    )


def fcc_ball(radius: float, a: float = A_LATTICE) -> np.ndarray:
    """fcc sites within `radius` of a lattice site at the origin, origin first."""
    m = int(np.ceil(radius / a)) + 1
    r = np.arange(-m, m + 1)
    n = np.stack(np.meshgrid(r, r, r, indexing="ij"), axis=-1).reshape(-1, 1, 3)
    sites = (a * (n + _FCC_BASIS[None, :, :])).reshape(-1, 3)
    d2 = np.sum(sites**2, axis=1)
    sites = sites[d2 <= radius * radius + 1e-9]
    d2 = np.sum(sites**2, axis=1)
    return np.ascontiguousarray(sites[np.argsort(d2, kind="stable")])


def dimer(r: float) -> np.ndarray:
    return np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])


def trimer(r: float) -> np.ndarray:
    """Equilateral triangle of side r in the xy plane."""
    return np.array(
        [[0.0, 0.0, 0.0], [r, 0.0, 0.0], [0.5 * r, 0.5 * np.sqrt(3.0) * r, 0.0]]
    )


def jitter(x: np.ndarray, sigma: float, seed: int) -> np.ndarray:
    """Gaussian displacement of every coordinate (numpy PCG64, seeded)."""
    rng = np.random.default_rng(seed)
    return x + sigma * rng.standard_normal(x.shape)


@dataclasses.dataclass
class Batch:
    """A ragged batch: wires concatenated atom-wise, in wire order.

    x      (N, 3) float64 positions, atoms of wire w at rows offset[w]..offset[w]+n[w]
    kind   (N,)   uint8   0 mobile, 1 left grip, 2 right grip
    offset (W,)   int64
    n      (W,)   int32
    L0, strain_rate, temperature, gamma (W,) float64; seed (W,) uint64
    """

    x: np.ndarray
    kind: np.ndarray
    offset: np.ndarray
    n: np.ndarray
    L0: np.ndarray
    strain_rate: np.ndarray
    temperature: np.ndarray
    gamma: np.ndarray
    seed: np.ndarray

    @property
    def n_atoms(self) -> int:
        return int(self.x.shape[0])

    @property
    def n_wires(self) -> int:
        return int(self.n.shape[0])

    def wire_slice(self, w: int) -> slice:
        o = int(self.offset[w])
        return slice(o, o + int(self.n[w]))


def pack(wires: list[Wire]) -> Batch:
    n = np.array([w.n for w in wires], dtype=np.int32)
    offset = np.zeros(len(wires), dtype=np.int64)
    if len(wires) > 1:
        offset[1:] = np.cumsum(n[:-1].astype(np.int64))
    return Batch(
        x=np.ascontiguousarray(np.concatenate([w.x for w in wires], axis=0)),
        kind=np.ascontiguousarray(np.concatenate([w.kind for w in wires])),
        offset=offset,
        n=n,
        L0=np.array([w.L0 for w in wires], dtype=np.float64),
        strain_rate=np.array([w.strain_rate for w in wires], dtype=np.float64),
        temperature=np.array([w.temperature for w in wires], dtype=np.float64),
        gamma=np.array([w.gamma for w in wires], dtype=np.float64),
        seed=np.array([w.seed for w in wires], dtype=np.uint64),
    )

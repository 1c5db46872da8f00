"""FP64 CPU oracle for the TB-SMA nanowire MD hot path (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline /
reference leg may import this package.  It shares no code with the CUDA
library: the arithmetic lives in ``tbsma_oracle.c`` (plain C, double
precision), wrapped here with ctypes over numpy arrays.

Parity pins (tests/test_oracle_*.py) tie every function to something other
than itself: closed forms for the dimer and trimer, the bulk fcc shell sum and
Au's experimental lattice constant, central finite differences of the energy,
invariances, brute force vs cell-list pair sets, NVE energy conservation, the
Ornstein-Uhlenbeck law of the O step, the dimer vibration period, Triton's
Philox4x32-10, the affine-strain derivative of the energy for Eq. 5, the
Nosé–Hoover invariants (free particles, extended energy at O(dt^2)), the
barostat's extended energy, target stress and a fixed-strain scan of the
zero-stress length, and scipy's connected components and per-plane counts
for the topology.  The tabulated EAM (tests/test_oracle_eam.py): exactness
for quadratics and the third-order error of its interpolant, closed-form
dimer and trimer energies and forces, the linear continuation of the
embedding, TB-SMA itself when the tables sample Eq. 1-2, finite
differences and invariances; its MD and stress (EamPotential,
tests/test_oracle_eam_md.py): a velocity-Verlet loop over its forces, the
strain derivative of its energy, O(dt^2) energy conservation with a smooth
table, and the TB-SMA trajectory when the tables sample Eq. 1-2.
"""

from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tbsma_oracle.c")
_LIB = os.path.join(_HERE, "libtbsma_oracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, IEEE semantics, OpenMP over wires)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", _LIB, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
        _declare(_lib)
    return _lib


class _Pot(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("A", "xi", "p", "q", "r0", "r_cut")] + [
        ("eam", ctypes.c_void_p)]


class _Md(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("r_skin", ctypes.c_double)]


class _Wire(ctypes.Structure):
    _fields_ = [
        ("L0", ctypes.c_double),
        ("strain_rate", ctypes.c_double),
        ("temperature", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("seed", ctypes.c_uint64),
    ]


class _Protocol(ctypes.Structure):
    _fields_ = [
        ("thermostat", ctypes.c_int),
        ("pull", ctypes.c_int),
        ("tau", ctypes.c_double),
        ("pull_step", ctypes.c_double),
        ("pull_interval", ctypes.c_int64),
        ("t_start", ctypes.c_double),
        ("ramp_steps", ctypes.c_int64),
        ("baro_tau", ctypes.c_double),
        ("baro_modulus", ctypes.c_double),
        ("baro_pressure", ctypes.c_double),
        ("baro_drag", ctypes.c_double),
        ("ramp_start", ctypes.c_int64),
    ]


_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_L = ctypes.c_long
_I64 = ctypes.c_int64
_U32 = ctypes.c_uint32
_U64 = ctypes.c_uint64


def _declare(L):
    L.or_mvv2e.restype = _D
    L.or_kb.restype = _D
    L.or_pairs_brute.argtypes = [_I, _P, _D, _P, _P, _L]
    L.or_pairs_brute.restype = _L
    L.or_pairs_cells.argtypes = [_I, _P, _D, _P, _P, _L]
    L.or_pairs_cells.restype = _L
    L.or_tbsma.argtypes = [_P, _I, _P, _P, _P, _P, _P, _P, _P, _P, _P]
    L.or_tbsma.restype = _D
    L.or_energy_forces.argtypes = [_P, _I, _P, _I, _P, _P, _P, _P, _P, _P, _P]
    L.or_energy_forces.restype = _D
    L.or_philox_many.argtypes = [_L, _P, _P, _P]
    L.or_normals_many.argtypes = [_L, _U64, _P, _U64, _U32, _P]
    L.or_init_velocities.argtypes = [_P, _I, _P, _U64, _D, _P]
    L.or_md_steps.argtypes = [_P, _P, _P, _I, _P, _P, _P, _P, _P, _I64, _I64, _D, _P, _P, _I]
    L.or_md_batch.argtypes = [_P, _P, _I, _P, _P, _P, _P, _P, _P, _P, _P, _I64, _I64, _D, _P, _P, _I]
    L.or_max_threads.restype = _I
    L.or_target_temperature.argtypes = [_P, _D, _I64]
    L.or_target_temperature.restype = _D
    L.or_md_steps_protocol.argtypes = [_P, _P, _P, _P, _I, _P, _P, _P, _P, _P, _I64, _I64, _D, _P,
                                       _P, _P, _I]
    L.or_md_batch_protocol.argtypes = [_P, _P, _P, _I, _P, _P, _P, _P, _P, _P, _P, _P, _I64, _I64,
                                       _D, _P, _P, _P, _I]
    L.or_observables.argtypes = [_P, _P, _P, _I, _P, _P, _P, _D, _I, _P]
    L.or_topology.argtypes = [_I, _P, _P, _D, _D, _L, _P, _P]
    L.or_topology.restype = _L
    L.or_eam_interp.argtypes = [_P, _I, _D, _D, _P]
    L.or_eam_interp.restype = _D
    L.or_eam_energy_forces.argtypes = [_P, _I, _P, _I, _P, _P, _P, _P, _P, _P, _P]
    L.or_eam_energy_forces.restype = _D
    L.or_eam_on_pairs.argtypes = [_P, _I, _P, _P, _P, _P, _P, _P, _P, _P, _P]
    L.or_eam_on_pairs.restype = _D


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


@dataclasses.dataclass(frozen=True)
class Potential:
    """TB-SMA parameters for Au (Table 1).

    r0 = 2.884 A: Table 1 prints 4.079 A in the r0 column, which is Au's fcc
    lattice constant; the TB-SMA r0 is the nearest-neighbour distance
    4.079/sqrt(2).  The hard cutoff r_cut = 5.8 A is stated after Eq. 3.
    """

    A: float = 0.2061
    xi: float = 1.790
    p: float = 10.229
    q: float = 4.036
    r0: float = 2.884
    r_cut: float = 5.8

    def _c(self):
        return _Pot(self.A, self.xi, self.p, self.q, self.r0, self.r_cut, None)


AU = Potential()
MASS_AU = 196.966569  # amu
R_SKIN = 0.29  # A, the HOOMD-Blue neighbour-list buffer in the benchmarks


def mvv2e() -> float:
    return lib().or_mvv2e()


def kb() -> float:
    return lib().or_kb()


def _f64(x):
    return np.ascontiguousarray(x, dtype=np.float64)


# ---------------------------------------------------------------- pair sets
def pairs(x: np.ndarray, rc: float, mode: str = "brute"):
    """CSR pair set (start, nbr) of all j != i with r_ij <= rc, ascending j."""
    x = _f64(x)
    n = x.shape[0]
    cap = 64 * n + 64
    while True:
        start = np.zeros(n + 1, dtype=np.int32)
        nbr = np.zeros(max(cap, 1), dtype=np.int32)
        f = lib().or_pairs_brute if mode == "brute" else lib().or_pairs_cells
        k = f(n, _ptr(x), rc, _ptr(start), _ptr(nbr), cap)
        if k >= 0:
            return start, nbr[:k].copy()
        cap *= 2


# --------------------------------------------------------- energy / forces
@dataclasses.dataclass
class Forces:
    E: float
    F: np.ndarray  # (n, 3) eV/A
    rho: np.ndarray
    eB: np.ndarray
    eR: np.ndarray
    w: np.ndarray  # per-atom 1/2 sum_j r_x,ij F_x,ij (eV)
    S: np.ndarray  # per-atom sum_j |f_ij| (eV/A)
    n_pairs: int


def tbsma(x: np.ndarray, pot: Potential = AU, brute_max: int = 2000) -> Forces:
    """Eq. 1-3 energy and forces (two passes), pairs from scratch."""
    x = _f64(x)
    n = x.shape[0]
    F = np.zeros((n, 3))
    rho, eB, eR, w, S = (np.zeros(n) for _ in range(5))
    npairs = ctypes.c_long(0)
    p = pot._c()
    E = lib().or_energy_forces(
        ctypes.byref(p), n, _ptr(x), brute_max, _ptr(F), _ptr(rho), _ptr(eB), _ptr(eR),
        _ptr(w), _ptr(S), ctypes.byref(npairs),
    )
    return Forces(E, F, rho, eB, eR, w, S, int(npairs.value))


def energy(x: np.ndarray, pot: Potential = AU, brute_max: int = 2000) -> float:
    x = _f64(x)
    p = pot._c()
    return lib().or_energy_forces(
        ctypes.byref(p), x.shape[0], _ptr(x), brute_max, None, None, None, None, None, None, None
    )


def tbsma_on_pairs(x, start, nbr, pot: Potential = AU) -> Forces:
    """Eq. 1-3 on a caller-given pair set (an EamPotential: its EAM)."""
    if isinstance(pot, EamPotential):
        return eam_on_pairs(x, start, nbr, pot.tab)
    x = _f64(x)
    n = x.shape[0]
    start = np.ascontiguousarray(start, dtype=np.int32)
    nbr = np.ascontiguousarray(nbr, dtype=np.int32)
    F = np.zeros((n, 3))
    rho, eB, eR, w, S = (np.zeros(n) for _ in range(5))
    p = pot._c()
    E = lib().or_tbsma(
        ctypes.byref(p), n, _ptr(x), _ptr(start), _ptr(nbr), _ptr(rho), _ptr(F), _ptr(eB),
        _ptr(eR), _ptr(w), _ptr(S),
    )
    return Forces(E, F, rho, eB, eR, w, S, int(nbr.shape[0]))


# ------------------------------------------------------------------ Philox
def philox4x32_10(ctr: np.ndarray, key: np.ndarray) -> np.ndarray:
    """ctr (n, 4) uint32, key (n, 2) uint32 -> (n, 4) uint32."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(np.broadcast_to(np.asarray(key, dtype=np.uint32).reshape(-1, 2),
                                               (ctr.shape[0], 2)))
    out = np.zeros_like(ctr)
    lib().or_philox_many(ctr.shape[0], _ptr(ctr), _ptr(key), _ptr(out))
    return out


def normals(seed: int, atoms: np.ndarray, step: int, tag: int) -> np.ndarray:
    """(n, 3) standard normals for atom indices `atoms` (Philox + Box-Muller)."""
    atoms = np.ascontiguousarray(atoms, dtype=np.uint32)
    out = np.zeros((atoms.shape[0], 3))
    lib().or_normals_many(atoms.shape[0], seed, _ptr(atoms), step, tag, _ptr(out))
    return out


# ---------------------------------------------------------------------- MD
def init_velocities(kind: np.ndarray, seed: int, T: float, mass: float = MASS_AU) -> np.ndarray:
    kind = np.ascontiguousarray(kind, dtype=np.uint8)
    n = kind.shape[0]
    v = np.zeros((n, 3))
    m = _Md(mass, R_SKIN)
    lib().or_init_velocities(ctypes.byref(m), n, _ptr(kind), seed, T, _ptr(v))
    return v


@dataclasses.dataclass
class WireState:
    """Mutable state of one wire for md_steps (positions (n,3), velocities (n,3))."""

    x: np.ndarray
    v: np.ndarray
    kind: np.ndarray
    L0: float
    strain_rate: float = 0.0
    temperature: float = 0.0
    gamma: float = 0.0
    seed: int = 0
    step: int = 0
    d_grip: float = 0.0
    n_rebuild: int = 0
    F: np.ndarray | None = None
    x_build: np.ndarray | None = None


def md_steps(st: WireState, n_steps: int, dt: float, pot: Potential = AU,
             mass: float = MASS_AU, r_skin: float = R_SKIN, brute_max: int = 2000) -> WireState:
    """Advance one wire by n_steps BAOAB steps in place (see tbsma_oracle.c)."""
    st.x = _f64(st.x)
    st.v = _f64(st.v)
    kind = np.ascontiguousarray(st.kind, dtype=np.uint8)
    if st.F is None:
        st.F = tbsma(st.x, pot, brute_max).F
    if st.x_build is None:
        st.x_build = st.x.copy()
    p, m = pot._c(), _Md(mass, r_skin)
    w = _Wire(st.L0, st.strain_rate, st.temperature, st.gamma, st.seed)
    dg = ctypes.c_double(st.d_grip)
    nr = ctypes.c_int64(st.n_rebuild)
    lib().or_md_steps(
        ctypes.byref(p), ctypes.byref(m), ctypes.byref(w), st.x.shape[0], _ptr(st.x), _ptr(st.v),
        _ptr(kind), _ptr(st.F), _ptr(st.x_build), st.step, n_steps, dt, ctypes.byref(dg),
        ctypes.byref(nr), brute_max,
    )
    st.step += n_steps
    st.d_grip = dg.value
    st.n_rebuild = int(nr.value)
    return st


def md_batch(x, v, kind, offset, count, L0, strain_rate, temperature, gamma, seed,
             step0: int, n_steps: int, dt: float, pot: Potential = AU, mass: float = MASS_AU,
             r_skin: float = R_SKIN, brute_max: int = 2000, F=None, x_build=None,
             d_grip=None, n_rebuild=None):
    """Advance a ragged batch of independent wires in place (OpenMP over wires).

    Returns (F, x_build, d_grip, n_rebuild) for continuation.
    """
    W = len(count)
    offset = np.ascontiguousarray(offset, dtype=np.int64)
    count = np.ascontiguousarray(count, dtype=np.int32)
    kind = np.ascontiguousarray(kind, dtype=np.uint8)
    if F is None:
        F = np.zeros_like(x)
        for w in range(W):
            s = slice(int(offset[w]), int(offset[w]) + int(count[w]))
            F[s] = tbsma(x[s], pot, brute_max).F
    if x_build is None:
        x_build = x.copy()
    if d_grip is None:
        d_grip = np.zeros(W)
    if n_rebuild is None:
        n_rebuild = np.zeros(W, dtype=np.int64)
    wires = (_Wire * W)(*[
        _Wire(float(L0[w]), float(strain_rate[w]), float(temperature[w]), float(gamma[w]),
              int(seed[w]))
        for w in range(W)
    ])
    p, m = pot._c(), _Md(mass, r_skin)
    lib().or_md_batch(
        ctypes.byref(p), ctypes.byref(m), W, wires, _ptr(offset), _ptr(count), _ptr(x), _ptr(v),
        _ptr(kind), _ptr(F), _ptr(x_build), step0, n_steps, dt, _ptr(d_grip), _ptr(n_rebuild),
        brute_max,
    )
    return F, x_build, d_grip, n_rebuild


@dataclasses.dataclass(frozen=True)
class Protocol:
    """Paper protocol mode (Methods, "Simulation details"); see or_md_steps_protocol.

    thermostat: "langevin" (B A O A B) or "nose_hoover" (period tau, fs);
    pull: "continuous" (strain rate) or "stepwise" (pull_step A per grip every
    pull_interval steps); temperature ramp from t_start (K) over ramp_steps
    (0: none).  The paper's values: Nosé–Hoover, 0.05 A every 10000 steps
    (20 ps at 2 fs), ramp from 0.01 K over 200000 steps (400 ps).
    """

    thermostat: str = "nose_hoover"
    pull: str = "stepwise"
    tau: float = 1000.0
    pull_step: float = 0.05
    pull_interval: int = 10000
    t_start: float = 0.01
    ramp_steps: int = 0
    baro_tau: float = 0.0  # fs, barostat period / 2 pi at modulus baro_modulus; 0 = off
    baro_modulus: float = 100.0 / 160.21766208  # 100 GPa in eV/A^3
    baro_pressure: float = 0.0  # target sigma_xx, eV/A^3
    baro_drag: float = 1.0  # barostat drag in units of 1/baro_tau
    ramp_start: int = 0  # first step of the ramp (t_start before it)

    def _c(self):
        th = {"langevin": 0, "nose_hoover": 1}[self.thermostat]
        pl = {"continuous": 0, "stepwise": 1}[self.pull]
        return _Protocol(th, pl, self.tau, self.pull_step, int(self.pull_interval), self.t_start,
                         int(self.ramp_steps), self.baro_tau, self.baro_modulus, self.baro_pressure,
                         self.baro_drag, int(self.ramp_start))


def target_temperature(proto: Protocol, T_w: float, step: int) -> float:
    return lib().or_target_temperature(ctypes.byref(proto._c()), T_w, int(step))


def md_steps_protocol(st: WireState, proto: Protocol, n_steps: int, dt: float,
                      nh: np.ndarray | None = None, pot: Potential = AU, mass: float = MASS_AU,
                      r_skin: float = R_SKIN, brute_max: int = 2000):
    """Advance one wire by n_steps protocol-mode steps in place.

    nh = [xi, eta, lambda, zeta] (the wire's Nosé–Hoover variable, its
    integral, the barostat's log-stretch and strain rate, in/out; zeros if
    None).  Returns (st, nh)."""
    st.x = _f64(st.x)
    st.v = _f64(st.v)
    kind = np.ascontiguousarray(st.kind, dtype=np.uint8)
    if st.F is None:
        st.F = tbsma(st.x, pot, brute_max).F
    if st.x_build is None:
        st.x_build = st.x.copy()
    nh = np.zeros(4) if nh is None else np.ascontiguousarray(nh, dtype=np.float64)
    p, m, r = pot._c(), _Md(mass, r_skin), proto._c()
    w = _Wire(st.L0, st.strain_rate, st.temperature, st.gamma, st.seed)
    dg = ctypes.c_double(st.d_grip)
    nr = ctypes.c_int64(st.n_rebuild)
    lib().or_md_steps_protocol(
        ctypes.byref(p), ctypes.byref(m), ctypes.byref(w), ctypes.byref(r), st.x.shape[0],
        _ptr(st.x), _ptr(st.v), _ptr(kind), _ptr(st.F), _ptr(st.x_build), st.step, n_steps, dt,
        ctypes.byref(dg), ctypes.byref(nr), _ptr(nh), brute_max,
    )
    st.step += n_steps
    st.d_grip = dg.value
    st.n_rebuild = int(nr.value)
    return st, nh


def md_batch_protocol(proto: Protocol, x, v, kind, offset, count, L0, strain_rate, temperature,
                      gamma, seed, step0: int, n_steps: int, dt: float, pot: Potential = AU,
                      mass: float = MASS_AU, r_skin: float = R_SKIN, brute_max: int = 2000,
                      F=None, x_build=None, d_grip=None, n_rebuild=None, nh=None):
    """md_batch in protocol mode; nh is (W, 4) [xi, eta, lambda, zeta] per wire (in/out).

    Returns (F, x_build, d_grip, n_rebuild, nh)."""
    W = len(count)
    offset = np.ascontiguousarray(offset, dtype=np.int64)
    count = np.ascontiguousarray(count, dtype=np.int32)
    kind = np.ascontiguousarray(kind, dtype=np.uint8)
    if F is None:
        F = np.zeros_like(x)
        for w in range(W):
            s = slice(int(offset[w]), int(offset[w]) + int(count[w]))
            F[s] = tbsma(x[s], pot, brute_max).F
    if x_build is None:
        x_build = x.copy()
    if d_grip is None:
        d_grip = np.zeros(W)
    if n_rebuild is None:
        n_rebuild = np.zeros(W, dtype=np.int64)
    if nh is None:
        nh = np.zeros((W, 4))
    wires = (_Wire * W)(*[
        _Wire(float(L0[w]), float(strain_rate[w]), float(temperature[w]), float(gamma[w]),
              int(seed[w]))
        for w in range(W)
    ])
    p, m, r = pot._c(), _Md(mass, r_skin), proto._c()
    lib().or_md_batch_protocol(
        ctypes.byref(p), ctypes.byref(m), ctypes.byref(r), W, wires, _ptr(offset), _ptr(count),
        _ptr(x), _ptr(v), _ptr(kind), _ptr(F), _ptr(x_build), step0, n_steps, dt, _ptr(d_grip),
        _ptr(n_rebuild), _ptr(nh), brute_max,
    )
    return F, x_build, d_grip, n_rebuild, nh


A_LATTICE = 4.079  # A, the fcc lattice constant of the wires (Table 1 column)


@dataclasses.dataclass
class Topology:
    connected: bool  # a left-grip and a right-grip atom share a cluster
    n_clusters: int
    neck: int  # smallest number of atoms in an axial slab between the grips
    neck_slab: int
    n_slabs: int
    label: np.ndarray  # component label (smallest atom index) of every atom


def topology(x: np.ndarray, kind: np.ndarray, pot: Potential = AU,
             slab: float = 0.5 * A_LATTICE) -> Topology:
    """Clusters of the interacting-pair graph and the neck (see or_topology)."""
    x = _f64(x)
    kind = np.ascontiguousarray(kind, dtype=np.uint8)
    n = x.shape[0]
    label = np.zeros(n, dtype=np.int32)
    out = np.zeros(5, dtype=np.int64)
    cap = 64 * n + 64
    while True:
        r = lib().or_topology(n, _ptr(x), _ptr(kind), pot.r_cut, slab, cap, _ptr(label),
                              _ptr(out))
        if r == 0:
            break
        if cap > 1024 * n + 1024:
            raise ValueError("a wire needs atoms of both grips")
        cap *= 4
    return Topology(bool(out[0]), int(out[1]), int(out[2]), int(out[3]), int(out[4]), label)


def max_threads() -> int:
    return lib().or_max_threads()


@dataclasses.dataclass
class Observables:
    e_pot: float
    e_kin: float
    temp: float
    sigma_xx: float  # eV/A^3
    virial_xx: float  # eV
    strain: float


def observables(st: WireState, pot: Potential = AU, mass: float = MASS_AU,
                brute_max: int = 2000) -> Observables:
    out = np.zeros(6)
    p, m = pot._c(), _Md(mass, R_SKIN)
    w = _Wire(st.L0, st.strain_rate, st.temperature, st.gamma, st.seed)
    kind = np.ascontiguousarray(st.kind, dtype=np.uint8)
    lib().or_observables(
        ctypes.byref(p), ctypes.byref(m), ctypes.byref(w), st.x.shape[0], _ptr(_f64(st.x)),
        _ptr(_f64(st.v)), _ptr(kind), st.d_grip, brute_max, _ptr(out),
    )
    return Observables(*[float(t) for t in out])


# ------------------------------------------------------------- tabulated EAM
class _Eam(ctypes.Structure):
    _fields_ = [("F", ctypes.c_void_p), ("n_rho", ctypes.c_int), ("d_rho", ctypes.c_double),
                ("f", ctypes.c_void_p), ("phi", ctypes.c_void_p), ("n_r", ctypes.c_int),
                ("d_r", ctypes.c_double), ("r_cut", ctypes.c_double)]


@dataclasses.dataclass
class EamTables:
    """EAM functions sampled on uniform grids: F(k d_rho) for k < len(F),
    f(k d_r) and phi(k d_r) for k < len(f); pairs with r <= r_cut interact.
    E = sum_i F(rho_i) + 1/2 sum_{i != j} phi(r_ij), rho_i = sum_j f(r_ij)."""

    F: np.ndarray
    d_rho: float
    f: np.ndarray
    phi: np.ndarray
    d_r: float
    r_cut: float

    def _c(self):
        self._keep = [_f64(self.F), _f64(self.f), _f64(self.phi)]
        assert self._keep[0].size >= 3 and self._keep[1].size == self._keep[2].size >= 3
        return _Eam(self._keep[0].ctypes.data, self._keep[0].size, self.d_rho,
                    self._keep[1].ctypes.data, self._keep[2].ctypes.data, self._keep[1].size,
                    self.d_r, self.r_cut)


class EamPotential:
    """A tabulated EAM in place of TB-SMA for every oracle function that takes
    a potential (md_steps, md_batch, md_steps_protocol, observables, ...):
    pairs within tab.r_cut; r0 only sets the hard-sphere volume of Eq. 5."""

    def __init__(self, tab: EamTables, r0: float = AU.r0):
        self.tab, self.r0, self.r_cut = tab, r0, tab.r_cut

    def _c(self):
        self._e = self.tab._c()  # kept alive with the struct that points to it
        return _Pot(0.0, 0.0, 0.0, 0.0, self.r0, self.r_cut,
                    ctypes.cast(ctypes.pointer(self._e), ctypes.c_void_p))


def eam_interp(y: np.ndarray, h: float, s) -> tuple[np.ndarray, np.ndarray]:
    """The tables' interpolant (cubic Hermite, finite-difference node slopes,
    straight-line continuation past the ends): value and derivative at s."""
    y = _f64(y)
    s = np.atleast_1d(np.asarray(s, dtype=np.float64))
    val, der = np.empty_like(s), np.empty_like(s)
    d = ctypes.c_double(0.0)
    for k, sk in enumerate(s):
        val[k] = lib().or_eam_interp(_ptr(y), y.size, h, float(sk), ctypes.byref(d))
        der[k] = d.value
    return val, der


def eam(x: np.ndarray, tab: EamTables, brute_max: int = 2000) -> Forces:
    """Tabulated EAM energy and forces (two passes), pairs from scratch;
    eB = F(rho_i), eR = 1/2 sum_j phi(r_ij)."""
    x = _f64(x)
    n = x.shape[0]
    F = np.zeros((n, 3))
    rho, eB, eR, w, S = (np.zeros(n) for _ in range(5))
    npairs = ctypes.c_long(0)
    t = tab._c()
    E = lib().or_eam_energy_forces(
        ctypes.byref(t), n, _ptr(x), brute_max, _ptr(F), _ptr(rho), _ptr(eB), _ptr(eR),
        _ptr(w), _ptr(S), ctypes.byref(npairs),
    )
    return Forces(E, F, rho, eB, eR, w, S, int(npairs.value))


def eam_energy(x: np.ndarray, tab: EamTables, brute_max: int = 2000) -> float:
    x = _f64(x)
    t = tab._c()
    return lib().or_eam_energy_forces(ctypes.byref(t), x.shape[0], _ptr(x), brute_max,
                                      None, None, None, None, None, None, None)


def eam_on_pairs(x, start, nbr, tab: EamTables) -> Forces:
    """Tabulated EAM on a caller-given pair set."""
    x = _f64(x)
    n = x.shape[0]
    start = np.ascontiguousarray(start, dtype=np.int32)
    nbr = np.ascontiguousarray(nbr, dtype=np.int32)
    F = np.zeros((n, 3))
    rho, eB, eR, w, S = (np.zeros(n) for _ in range(5))
    t = tab._c()
    E = lib().or_eam_on_pairs(ctypes.byref(t), n, _ptr(x), _ptr(start), _ptr(nbr), _ptr(rho),
                              _ptr(F), _ptr(eB), _ptr(eR), _ptr(w), _ptr(S))
    return Forces(E, F, rho, eB, eR, w, S, int(nbr.shape[0]))

"""ctypes binding of libtbsma.so (include/tbsma.h).

Argument marshalling only: every step of the MD path runs in the CUDA
library.  Device memory and streams come from PyTorch.  There is no CPU
fallback: if the compiled library is missing or fails to load, the first
call that needs it raises.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtbsma.so")

FP64 = 0
MIXED = 1

STATUS_NAMES = {
    0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "EOVERFLOW", 5: "ETIMEOUT", 6: "EWIRE",
    7: "ESTATE",
}
WIRE_NONFINITE, WIRE_NBR_OVERFLOW, WIRE_CELL_OVERFLOW, WIRE_RANGE = 1, 2, 4, 8
WIRE_GRID_CLAMP = 16  # not a fault: the wire's cell grid is grown at the next status read
PHASES = ("integrate", "plan", "rebuild", "density", "force", "kick")  # tbsma_step_profile


class TbsmaError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: TBSMA_{STATUS_NAMES.get(status, status)} {detail}".rstrip())


class Params(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("A", "xi", "p", "q", "r0", "r_cut", "r_skin", "mass")]


def au_params(**over) -> Params:
    """TB-SMA Au (Table 1, r0 read as the nearest-neighbour distance 2.884 A),
    r_cut 5.8 A, list skin 0.29 A, Au mass 196.966569 amu."""
    d = dict(A=0.2061, xi=1.790, p=10.229, q=4.036, r0=2.884, r_cut=5.8, r_skin=0.29,
             mass=196.966569)
    d.update(over)
    return Params(**d)


class WireC(ctypes.Structure):
    _fields_ = [
        ("atom_offset", ctypes.c_int64),
        ("n_atoms", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("L0", ctypes.c_double),
        ("strain_rate", ctypes.c_double),
        ("temperature", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("seed", ctypes.c_uint64),
    ]


class ObsC(ctypes.Structure):
    _fields_ = [
        ("step", ctypes.c_int64),
        ("strain", ctypes.c_double),
        ("e_pot", ctypes.c_double),
        ("e_kin", ctypes.c_double),
        ("temp", ctypes.c_double),
        ("sigma_xx", ctypes.c_double),
        ("virial_xx", ctypes.c_double),
        ("n_rebuilds", ctypes.c_int32),
        ("status", ctypes.c_int32),
    ]


class FCheckC(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("max_err_scaled", "max_err_raw", "norm_err", "max_abs_err")]


_P = ctypes.c_void_p
_lib = None

# (name, restype, argtypes) of every entry point declared in include/tbsma.h
class ProtocolC(ctypes.Structure):
    """tbsma_protocol (include/tbsma.h)."""

    _fields_ = [
        ("thermostat", ctypes.c_int32),
        ("pull", ctypes.c_int32),
        ("tau_fs", ctypes.c_double),
        ("pull_step", ctypes.c_double),
        ("pull_interval", ctypes.c_int64),
        ("t_start", ctypes.c_double),
        ("ramp_steps", ctypes.c_int64),
        ("baro_tau_fs", ctypes.c_double),
        ("baro_modulus", ctypes.c_double),
        ("baro_pressure", ctypes.c_double),
        ("baro_drag", ctypes.c_double),
        ("ramp_start", ctypes.c_int64),
    ]


class TopologyC(ctypes.Structure):
    """tbsma_topology (include/tbsma.h)."""

    _fields_ = [(k, ctypes.c_int32) for k in ("connected", "n_clusters", "neck", "neck_slab",
                                                 "n_slabs", "status")]


class WireStateC(ctypes.Structure):
    """tbsma_wire_state (include/tbsma.h)."""

    _fields_ = [("d_grip", ctypes.c_double), ("xi", ctypes.c_double), ("eta", ctypes.c_double),
                ("log_stretch", ctypes.c_double), ("stretch_rate", ctypes.c_double),
                ("n_rebuilds", ctypes.c_int32),
                ("status", ctypes.c_uint32)]


class EamC(ctypes.Structure):
    """tbsma_eam (include/tbsma.h)."""

    _fields_ = [("F", ctypes.c_void_p), ("n_rho", ctypes.c_int32), ("d_rho", ctypes.c_double),
                ("f", ctypes.c_void_p), ("phi", ctypes.c_void_p), ("n_r", ctypes.c_int32),
                ("d_r", ctypes.c_double)]


THERMOSTATS = {"langevin": 0, "nose_hoover": 1}
BARO_MODULUS = 100.0 / 160.21766208  # 100 GPa in eV/A^3: the barostat's reference modulus
PULLS = {"continuous": 0, "stepwise": 1}
STEP_MODES = {"auto": 0, "graph": 1, "persistent": 2}

SIGNATURES = [
    ("tbsma_init", ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int32, _P, _P, _P, _P, _P, _P]),
    ("tbsma_init_velocities", ctypes.c_int, [_P]),
    ("tbsma_build_neighbors", ctypes.c_int, [_P, ctypes.c_int32, _P]),
    ("tbsma_compute_forces", ctypes.c_int, [_P, _P, _P]),
    ("tbsma_atom_energies", ctypes.c_int, [_P, _P, _P]),
    ("tbsma_step_nvt_pull", ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_double]),
    ("tbsma_reduce_observables", ctypes.c_int, [_P, _P]),
    ("tbsma_step_observe", ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_double, _P]),
    ("tbsma_force_check", ctypes.c_int, [_P, _P]),
    ("tbsma_upload_state", ctypes.c_int, [_P, _P, _P]),
    ("tbsma_download_state", ctypes.c_int, [_P, _P, _P]),
    ("tbsma_get_wire_status", ctypes.c_int, [_P, _P]),
    ("tbsma_nbr_capacity", ctypes.c_int32, [_P]),
    ("tbsma_get_rebuild_chains", ctypes.c_int, [_P, _P]),
    ("tbsma_get_neighbors", ctypes.c_int, [_P, _P, _P, ctypes.c_int32]),
    ("tbsma_set_launch", ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32]),
    ("tbsma_run_pass", ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32]),
    ("tbsma_step_profile", ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_double, _P]),
    ("tbsma_get_rebuild_stats", ctypes.c_int, [_P, _P]),
    ("tbsma_set_protocol", ctypes.c_int, [_P, _P]),
    ("tbsma_get_thermostat", ctypes.c_int, [_P, _P, _P]),
    ("tbsma_get_barostat", ctypes.c_int, [_P, _P, _P]),
    ("tbsma_set_eam", ctypes.c_int, [_P, _P]),
    ("tbsma_eam_cubics", ctypes.c_int, [_P, ctypes.c_int32, _P]),
    ("tbsma_wire_topology", ctypes.c_int, [_P, _P, _P]),
    ("tbsma_set_wait_limit", ctypes.c_int, [_P, ctypes.c_int32]),
    ("tbsma_set_step_mode", ctypes.c_int, [_P, ctypes.c_int32, _P]),
    ("tbsma_set_pair_lanes", ctypes.c_int, [_P, ctypes.c_int32]),
    ("tbsma_save_state", ctypes.c_int, [_P, _P, _P, _P, _P]),
    ("tbsma_restore_state", ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int64]),
    ("tbsma_philox4x32_10", ctypes.c_int, [_P, _P, ctypes.c_int64, _P, _P]),
    ("tbsma_normals", ctypes.c_int, [ctypes.c_uint64, _P, ctypes.c_int64, ctypes.c_int64,
                                     ctypes.c_uint32, ctypes.c_int, _P, _P]),
    ("tbsma_forces_noalloc", ctypes.c_int, [_P, ctypes.c_int32, _P, _P, _P]),
    ("tbsma_last_error", ctypes.c_char_p, [_P]),
    ("tbsma_destroy", None, [_P]),
]


def lib() -> ctypes.CDLL:
    """Load libtbsma.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"{LIB_PATH} is missing; build it with `python -m paper_1311_3890_b300.build`")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _stream_ptr(stream=None):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _hptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.dtype == np.float64 and a.flags.c_contiguous
        return a.ctypes.data_as(ctypes.c_void_p)
    return ctypes.c_void_p(a.data_ptr())


class Engine:
    """A batch of wires on one GPU, driven through the C ABI.

    batch: an inputs.Batch (positions (N,3) float64, kind, per-wire table).
    precision: "mixed" or "fp64".
    """

    def __init__(self, batch, precision: str = "mixed", params: Params | None = None,
                 device: str = "cuda", stream=None):
        import torch

        self.torch = torch
        self.device = torch.device(device)
        self.batch = batch
        self.N = int(batch.n_atoms)
        self.W = int(batch.n_wires)
        self.precision = MIXED if precision == "mixed" else FP64
        self.params = params if params is not None else au_params()
        self.stream = stream
        self.ctx = ctypes.c_void_p()
        # SoA device state: x[0:N] = x coords, x[N:2N] = y, x[2N:3N] = z
        self.x = torch.from_numpy(np.ascontiguousarray(batch.x.T).reshape(-1)).to(self.device)
        self.v = torch.zeros(3 * self.N, dtype=torch.float64, device=self.device)
        self.kind = torch.from_numpy(np.ascontiguousarray(batch.kind, dtype=np.uint8)).to(self.device)
        wires = (WireC * self.W)()
        for w in range(self.W):
            wires[w] = WireC(int(batch.offset[w]), int(batch.n[w]), 0, float(batch.L0[w]),
                             float(batch.strain_rate[w]), float(batch.temperature[w]),
                             float(batch.gamma[w]), int(batch.seed[w]))
        self._wires = wires
        st = lib().tbsma_init(ctypes.byref(self.params), self.precision, self.W, wires,
                              _ptr(self.x), _ptr(self.v), _ptr(self.kind),
                              _stream_ptr(stream), ctypes.byref(self.ctx))
        if st != 0:
            detail = ""
            if self.ctx:
                detail = lib().tbsma_last_error(self.ctx).decode()
                lib().tbsma_destroy(self.ctx)
                self.ctx = ctypes.c_void_p()
            raise TbsmaError(st, "tbsma_init", detail)

    # ----------------------------------------------------------- plumbing
    def _check(self, st, where):
        if st != 0:
            raise TbsmaError(st, where, lib().tbsma_last_error(self.ctx).decode())

    def close(self):
        if getattr(self, "ctx", None):
            lib().tbsma_destroy(self.ctx)
            self.ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ the path
    def init_velocities(self):
        self._check(lib().tbsma_init_velocities(self.ctx), "tbsma_init_velocities")

    def build_neighbors(self, force_all: bool = False) -> int:
        n = ctypes.c_int32(0)
        self._check(lib().tbsma_build_neighbors(self.ctx, int(force_all), ctypes.byref(n)),
                    "tbsma_build_neighbors")
        return int(n.value)

    def step(self, n_steps: int, dt: float = 2.0, check: bool = True) -> int:
        st = lib().tbsma_step_nvt_pull(self.ctx, int(n_steps), float(dt))
        if check:
            self._check(st, "tbsma_step_nvt_pull")
        return st

    def forces(self, f32: bool = True, f64: bool = True):
        """(F_mixed float32 (N,3) or None, F_fp64 float64 (N,3) or None)."""
        t = self.torch
        a = t.empty(3 * self.N, dtype=t.float32, device=self.device) if f32 else None
        b = t.empty(3 * self.N, dtype=t.float64, device=self.device) if f64 else None
        self._check(lib().tbsma_compute_forces(self.ctx, _ptr(a), _ptr(b)), "tbsma_compute_forces")
        return (a.view(3, self.N).T if f32 else None, b.view(3, self.N).T if f64 else None)

    def atom_energies(self):
        t = self.torch
        e = t.empty(self.N, dtype=t.float64, device=self.device)
        w = t.empty(self.N, dtype=t.float64, device=self.device)
        self._check(lib().tbsma_atom_energies(self.ctx, _ptr(e), _ptr(w)), "tbsma_atom_energies")
        return e, w

    def observables(self, check: bool = True) -> np.ndarray:
        out = (ObsC * self.W)()
        st = lib().tbsma_reduce_observables(self.ctx, out)
        if check:
            self._check(st, "tbsma_reduce_observables")
        return np.ctypeslib.as_array(out).copy()

    def step_observe(self, n_steps: int, dt: float = 2.0, check: bool = True) -> np.ndarray:
        """step(n_steps, dt), then observables(), in one call
        (tbsma_step_observe): the same trajectory and bitwise the same
        report, the report's pair passes folded into the last step in graph
        replays."""
        out = (ObsC * self.W)()
        st = lib().tbsma_step_observe(self.ctx, int(n_steps), float(dt), out)
        if check:
            self._check(st, "tbsma_step_observe")
        return np.ctypeslib.as_array(out).copy()

    def force_check(self) -> np.ndarray:
        out = (FCheckC * self.W)()
        self._check(lib().tbsma_force_check(self.ctx, out), "tbsma_force_check")
        return np.ctypeslib.as_array(out).copy()

    def upload(self, x_host=None, v_host=None):
        """x_host, v_host: host float64 arrays of 3N (SoA); pinned torch tensors or numpy."""
        self._check(lib().tbsma_upload_state(self.ctx, _hptr(x_host), _hptr(v_host)),
                    "tbsma_upload_state")

    def download(self, x_host=None, v_host=None):
        self._check(lib().tbsma_download_state(self.ctx, _hptr(x_host), _hptr(v_host)),
                    "tbsma_download_state")

    def wire_status(self) -> np.ndarray:
        out = np.zeros(self.W, dtype=np.int32)
        self._check(lib().tbsma_get_wire_status(self.ctx, out.ctypes.data_as(ctypes.c_void_p)),
                    "tbsma_get_wire_status")
        return out

    def neighbors(self):
        t = self.torch
        cap = lib().tbsma_nbr_capacity(self.ctx)
        n = t.empty(self.N, dtype=t.int32, device=self.device)
        nb = t.empty(self.N * cap, dtype=t.int32, device=self.device)
        self._check(lib().tbsma_get_neighbors(self.ctx, _ptr(n), _ptr(nb), cap), "tbsma_get_neighbors")
        return n, nb.view(self.N, cap)

    def rebuild_chains(self) -> int:
        """Launches of the four-kernel list-rebuild chain so far (launch accounting)."""
        n = ctypes.c_int64(0)
        self._check(lib().tbsma_get_rebuild_chains(self.ctx, ctypes.byref(n)),
                    "tbsma_get_rebuild_chains")
        return int(n.value)

    def rebuild_stats(self) -> dict:
        """List-build accounting since init (tbsma_get_rebuild_stats): chain
        launches, wires rebuilt and atoms rebuilt."""
        out = np.zeros(3, dtype=np.int64)
        self._check(lib().tbsma_get_rebuild_stats(self.ctx, out.ctypes.data_as(ctypes.c_void_p)),
                    "tbsma_get_rebuild_stats")
        return {"chains": int(out[0]), "wires": int(out[1]), "atoms": int(out[2])}

    def step_profile(self, n_steps: int, dt: float = 2.0) -> dict:
        """n_steps steps enqueued directly with an event after each phase
        (tbsma_step_profile): summed ms per phase."""
        out = np.zeros(len(PHASES))
        self._check(lib().tbsma_step_profile(self.ctx, int(n_steps), float(dt),
                                             out.ctypes.data_as(ctypes.c_void_p)),
                    "tbsma_step_profile")
        return dict(zip(PHASES, (float(v) for v in out)))

    def set_launch(self, block_threads: int, window_atoms: int):
        """Pair-pass tile size (atoms per block) and shared-memory window (atoms)."""
        self._check(lib().tbsma_set_launch(self.ctx, block_threads, window_atoms), "tbsma_set_launch")

    def set_protocol(self, thermostat: str = "nose_hoover", pull: str = "stepwise",
                     tau_fs: float = 1000.0, pull_step: float = 0.05, pull_interval: int = 10000,
                     t_start: float = 0.01, ramp_steps: int = 0, baro_tau_fs: float = 0.0,
                     baro_modulus: float = BARO_MODULUS, baro_pressure: float = 0.0,
                     baro_drag: float = 1.0, ramp_start: int = 0):
        """Paper protocol mode (tbsma_set_protocol); the defaults are the paper's
        Nosé–Hoover thermostat and 0.05 A grip steps every 10000 steps, no ramp,
        no barostat (baro_tau_fs > 0 turns on the axial Nosé–Hoover barostat;
        baro_modulus and baro_pressure in eV/A^3, baro_drag in 1/baro_tau_fs);
        the ramp, when on, starts at step ramp_start (t_start before it)."""
        p = ProtocolC(THERMOSTATS[thermostat], PULLS[pull], tau_fs, pull_step, int(pull_interval),
                      t_start, int(ramp_steps), baro_tau_fs, baro_modulus, baro_pressure,
                      baro_drag, int(ramp_start))
        self._check(lib().tbsma_set_protocol(self.ctx, ctypes.byref(p)), "tbsma_set_protocol")
        self.protocol = dict(thermostat=thermostat, pull=pull, tau_fs=tau_fs, pull_step=pull_step,
                             pull_interval=int(pull_interval), t_start=t_start,
                             ramp_steps=int(ramp_steps), baro_tau_fs=baro_tau_fs,
                             baro_modulus=baro_modulus, baro_pressure=baro_pressure,
                             baro_drag=baro_drag, ramp_start=int(ramp_start))

    def set_eam(self, F=None, d_rho: float = 0.0, f=None, phi=None, d_r: float = 0.0,
                r_cut: float | None = None):
        """Tabulated EAM (tbsma_set_eam): F sampled at k d_rho, f and phi at
        k d_r; F=None returns to TB-SMA.  Pairs interact within the context's
        r_cut (params); a table set's own r_cut, if given, must equal it."""
        if r_cut is not None and r_cut != self.params.r_cut:
            raise ValueError(f"the tables' r_cut {r_cut} differs from the context's {self.params.r_cut}")
        if F is None:
            self._check(lib().tbsma_set_eam(self.ctx, None), "tbsma_set_eam")
            return
        keep = [np.ascontiguousarray(a, dtype=np.float64) for a in (F, f, phi)]
        if keep[1].size != keep[2].size:
            raise ValueError("f and phi need the same number of samples")
        t = EamC(keep[0].ctypes.data, keep[0].size, float(d_rho), keep[1].ctypes.data,
                 keep[2].ctypes.data, keep[1].size, float(d_r))
        self._check(lib().tbsma_set_eam(self.ctx, ctypes.byref(t)), "tbsma_set_eam")

    def set_eam_setfl(self, path: str, element=0):
        """set_eam from one element of a DYNAMO setfl file (eam_files.read_setfl);
        the file's cutoff and mass must equal the context's r_cut and mass."""
        from .eam_files import read_setfl

        t = read_setfl(path, element)
        if abs(t["mass"] - self.params.mass) > 1e-6 * self.params.mass:
            raise ValueError(f"the file's mass {t['mass']} differs from the context's {self.params.mass}")
        self.set_eam(t["F"], t["d_rho"], t["f"], t["phi"], t["d_r"], r_cut=t["r_cut"])

    def thermostat(self):
        """(xi, eta) per wire, numpy arrays (tbsma_get_thermostat)."""
        xi = np.zeros(self.W)
        eta = np.zeros(self.W)
        self._check(lib().tbsma_get_thermostat(self.ctx, xi.ctypes.data_as(ctypes.c_void_p),
                                               eta.ctypes.data_as(ctypes.c_void_p)),
                    "tbsma_get_thermostat")
        return xi, eta

    def barostat(self):
        """(lambda, zeta) per wire: the barostat's axial log-stretch and strain
        rate (1/fs), numpy arrays (tbsma_get_barostat)."""
        lam = np.zeros(self.W)
        zeta = np.zeros(self.W)
        self._check(lib().tbsma_get_barostat(self.ctx, lam.ctypes.data_as(ctypes.c_void_p),
                                             zeta.ctypes.data_as(ctypes.c_void_p)),
                    "tbsma_get_barostat")
        return lam, zeta

    def topology(self, labels: bool = False):
        """Per-wire rupture and neck (tbsma_wire_topology): dict of numpy arrays
        connected, n_clusters, neck, neck_slab, n_slabs, status; with
        labels=True also the per-atom cluster labels (cuda int32 tensor)."""
        out = (TopologyC * self.W)()
        lab = self.torch.empty(self.N, dtype=self.torch.int32, device=self.device) if labels else None
        self._check(lib().tbsma_wire_topology(self.ctx, out, _ptr(lab) if labels else None),
                    "tbsma_wire_topology")
        res = {k: np.array([getattr(o, k) for o in out], dtype=np.int32)
               for k, _ in TopologyC._fields_}
        res["connected"] = res["connected"].astype(bool)
        if labels:
            res["labels"] = lab
        return res

    def set_wait_limit(self, steps: int):
        """Bound of the topology's union-find walks (a failure-detection test hook)."""
        self._check(lib().tbsma_set_wait_limit(self.ctx, int(steps)), "tbsma_set_wait_limit")

    def set_step_mode(self, mode: str = "auto") -> int:
        """How steps run (tbsma_set_step_mode): "auto", "graph" or
        "persistent"; returns the blocks the persistent step kernel would use
        in this context (0: it cannot run it)."""
        b = ctypes.c_int32(0)
        self._check(lib().tbsma_set_step_mode(self.ctx, STEP_MODES[mode], ctypes.byref(b)),
                    "tbsma_set_step_mode")
        return int(b.value)

    def set_pair_lanes(self, lanes: int = 1):
        """Threads per atom in the MIXED pair passes (tbsma_set_pair_lanes):
        1 (default), 2 or 4 (bitwise the same results)."""
        self._check(lib().tbsma_set_pair_lanes(self.ctx, int(lanes)), "tbsma_set_pair_lanes")

    def save(self, path: str):
        """Checkpoint into directory `path` (tbsma_save_state): header.json and
        raw little-endian float64 SoA arrays x.f64, v.f64 (3N each)."""
        import json
        import os

        os.makedirs(path, exist_ok=True)
        x = np.empty(3 * self.N)
        v = np.empty(3 * self.N)
        ws = (WireStateC * self.W)()
        step = ctypes.c_int64(0)
        self._check(lib().tbsma_save_state(self.ctx, x.ctypes.data_as(ctypes.c_void_p),
                                           v.ctypes.data_as(ctypes.c_void_p), ws,
                                           ctypes.byref(step)), "tbsma_save_state")
        x.astype("<f8").tofile(os.path.join(path, "x.f64"))
        v.astype("<f8").tofile(os.path.join(path, "v.f64"))
        header = {
            "format": "tbsma-checkpoint-1", "n_atoms": self.N, "n_wires": self.W,
            "precision": "mixed" if self.precision == MIXED else "fp64", "step": int(step.value),
            "protocol": getattr(self, "protocol", None),
            "wires": [{k: getattr(w, k) for k, _ in WireStateC._fields_} for w in ws],
        }
        with open(os.path.join(path, "header.json"), "w") as f:
            json.dump(header, f, indent=1)

    def load(self, path: str):
        """Resume from a checkpoint written by save() for the same batch layout
        (re-applies its protocol first, then tbsma_restore_state)."""
        import json
        import os

        with open(os.path.join(path, "header.json")) as f:
            header = json.load(f)
        if header.get("format") != "tbsma-checkpoint-1":
            raise ValueError("not a tbsma checkpoint")
        if header["n_atoms"] != self.N or header["n_wires"] != self.W:
            raise ValueError("checkpoint of a different batch layout")
        if header.get("protocol"):
            self.set_protocol(**header["protocol"])
        x = np.fromfile(os.path.join(path, "x.f64"), dtype="<f8").astype(np.float64)
        v = np.fromfile(os.path.join(path, "v.f64"), dtype="<f8").astype(np.float64)
        ws = (WireStateC * self.W)()
        for w, d in zip(ws, header["wires"]):
            for k, _ in WireStateC._fields_:
                setattr(w, k, d.get(k, 0.0) if k in ("log_stretch", "stretch_rate") else d[k])
        self._check(lib().tbsma_restore_state(self.ctx, x.ctypes.data_as(ctypes.c_void_p),
                                              v.ctypes.data_as(ctypes.c_void_p), ws,
                                              int(header["step"])), "tbsma_restore_state")

    def run_pass(self, which: int, reps: int = 1):
        """Enqueue `reps` launches of pass 1 (density) or 2 (force) alone."""
        self._check(lib().tbsma_run_pass(self.ctx, which, reps), "tbsma_run_pass")

    # ------------------------------------------------------------- views
    def positions(self) -> np.ndarray:
        return self.x.view(3, self.N).T.cpu().numpy()

    def velocities(self) -> np.ndarray:
        return self.v.view(3, self.N).T.cpu().numpy()


def eam_cubics(samples) -> np.ndarray:
    """The per-interval cubic coefficients (n-1, 4) tbsma_set_eam derives
    from a sample table (host only; tbsma_eam_cubics)."""
    y = np.ascontiguousarray(samples, dtype=np.float64)
    out = np.empty((max(y.size - 1, 0), 4))
    st = lib().tbsma_eam_cubics(_hptr(y), y.size, _hptr(out))
    if st != 0:
        raise TbsmaError(st, "tbsma_eam_cubics")
    return out


def philox4x32_10(ctr, key, stream=None):
    """ctr (n,4) int32 cuda tensor (bit patterns), key (n,2) -> (n,4) int32 bits."""
    import torch

    out = torch.empty_like(ctr)
    st = lib().tbsma_philox4x32_10(_ptr(ctr), _ptr(key), ctr.shape[0], _ptr(out), _stream_ptr(stream))
    if st != 0:
        raise TbsmaError(st, "tbsma_philox4x32_10")
    return out


def normals(seed: int, atoms, step: int, tag: int, precision: str = "fp64", stream=None):
    """(n,3) float64 cuda tensor of the thermostat's Gaussian triples."""
    import torch

    n = atoms.shape[0]
    out = torch.empty((n, 3), dtype=torch.float64, device=atoms.device)
    st = lib().tbsma_normals(seed, _ptr(atoms), n, step, tag,
                             MIXED if precision == "mixed" else FP64, _ptr(out), _stream_ptr(stream))
    if st != 0:
        raise TbsmaError(st, "tbsma_normals")
    return out

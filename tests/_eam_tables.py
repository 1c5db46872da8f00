"""EAM tables for the tests: inputs of both the oracle and the CUDA path.

An EAM potential enters the library as samples of F(rho), f(r) and phi(r)
on uniform grids; these helpers sample two analytic sets.

* tbsma_sampled: the TB-SMA functions of Table 1 in EAM form,
  f = xi^2 e^{-2q s}, phi = 2 A e^{-p s}, F = -sqrt(rho), s = r/r0 - 1.
* synthetic: an Au-like set whose embedding is not a square root,
  F = -c sqrt(rho) + d rho^2, with f and phi exponentials tapered
  smoothly to zero at r_cut, so that every term of the EAM force
  (phi', F'(rho_i) f', F'(rho_j) f') carries its own shape.
"""

import numpy as np

A, XI, P, Q, R0, R_CUT = 0.2061, 1.790, 10.229, 4.036, 2.884, 5.8


def _grid(r_max: float, d: float) -> np.ndarray:
    return np.arange(int(np.ceil(r_max / d)) + 1) * d


def tbsma_sampled(d_r: float = 0.002, d_rho: float = 0.005, rho_max: float = 120.0):
    r = _grid(R_CUT + 0.05, d_r)
    s = r / R0 - 1.0
    f = XI * XI * np.exp(-2.0 * Q * s)
    phi = 2.0 * A * np.exp(-P * s)
    rho = _grid(rho_max, d_rho)
    F = -np.sqrt(rho)
    return dict(F=F, d_rho=d_rho, f=f, phi=phi, d_r=d_r, r_cut=R_CUT)


def _taper(r, r_s, r_c):
    t = np.clip((r_c - r) / (r_c - r_s), 0.0, 1.0)
    return t * t * t * (6 * t * t - 15 * t + 10)


def synthetic(d_r: float = 0.002, d_rho: float = 0.01, rho_max: float = 60.0):
    r_c = R_CUT
    r = _grid(r_c + 0.05, d_r)
    tap = _taper(r, 4.6, r_c)
    f = 1.9 * np.exp(-5.6 * (r / R0 - 1.0)) * tap
    phi = 0.55 * np.exp(-9.1 * (r / R0 - 1.0)) * tap
    rho = _grid(rho_max, d_rho)
    F = -1.05 * np.sqrt(rho) + 4.0e-4 * rho * rho
    return dict(F=F, d_rho=d_rho, f=f, phi=phi, d_r=d_r, r_cut=r_c)

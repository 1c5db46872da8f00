"""The oracle's MD, observables and stress with a tabulated EAM in place of
TB-SMA (oracle.EamPotential), pinned to things other than themselves: a
velocity-Verlet loop written here over the EAM forces, the strain
derivative of the EAM energy (Eq. 5 at T = 0), energy conservation with a
smooth table, and the TB-SMA trajectory when the tables sample Eq. 1-2."""

import math

import numpy as np
import pytest

from inputs import fcc_wire, jitter
from tests._eam_tables import synthetic, tbsma_sampled


def _pot(orc, d):
    return orc.EamPotential(orc.EamTables(**d))


def test_nve_steps_equal_a_velocity_verlet_loop(orc):
    """gamma = 0, no pull: the BAOAB step is velocity Verlet; 40 steps of the
    oracle's MD equal a loop over orc.eam forces (B, A, A, B) written here."""
    T = synthetic()
    pot = _pot(orc, T)
    w = fcc_wire(2.0, 2.0)
    x0 = jitter(w.x, 0.05, 1)
    v0 = np.random.default_rng(2).normal(scale=2e-3, size=x0.shape)
    v0[w.kind > 0] = 0.0
    st = orc.WireState(x=x0.copy(), v=v0.copy(), kind=w.kind, L0=w.L0)
    orc.md_steps(st, 40, 2.0, pot=pot, brute_max=10**6)
    m = orc.MASS_AU * orc.mvv2e()
    mob = w.kind == 0
    x, v = x0.copy(), v0.copy()
    tab = orc.EamTables(**T)
    F = orc.eam(x, tab, brute_max=10**6).F
    for _ in range(40):
        v[mob] += 0.5 * 2.0 * F[mob] / m
        x[mob] += 0.5 * 2.0 * v[mob]
        x[mob] += 0.5 * 2.0 * v[mob]
        F = orc.eam(x, tab, brute_max=10**6).F
        v[mob] += 0.5 * 2.0 * F[mob] / m
    assert np.max(np.abs(st.x - x)) < 1e-11
    assert np.max(np.abs(st.v - v)) < 1e-13
    assert np.max(np.abs(st.x - x0)) > 1e-3  # the atoms did move


def test_virial_stress_is_strain_derivative_of_eam_energy(orc):
    """At T = 0, V sigma_xx = sum_i 1/2 sum_j r_x,ij F_x,ij = dE/d(eps) under
    x -> (1 + eps) x, with the EAM's pair forces (a wrong factor on the
    embedding terms or on phi fails)."""
    T = synthetic()
    pot = _pot(orc, T)
    tab = orc.EamTables(**T)
    w = fcc_wire(2.0, 3.0)
    x = jitter(w.x, 0.03, seed=2)
    st = orc.WireState(x=x.copy(), v=np.zeros_like(x), kind=w.kind, L0=w.L0)
    ob = orc.observables(st, pot=pot)
    h = 1e-5

    def e(eps):
        y = x.copy()
        y[:, 0] *= 1 + eps
        return orc.eam_energy(y, tab)

    dE = (-e(2 * h) + 8 * e(h) - 8 * e(-h) + e(-2 * h)) / (12 * h)
    assert ob.virial_xx == pytest.approx(dE, rel=1e-6, abs=1e-6)
    V = w.n * 4 / 3 * math.pi * (orc.AU.r0 / 2) ** 3
    assert ob.sigma_xx == pytest.approx(ob.virial_xx / V, rel=1e-12)
    assert ob.e_pot == pytest.approx(orc.eam_energy(x, tab), rel=1e-14)


def test_nve_energy_is_conserved_with_a_smooth_table(orc):
    """The synthetic set is tapered to zero at r_cut (C2), so nothing jumps:
    over 1 ps of NVE from 300 K (the Au lattice is not this set's minimum:
    the wire relaxes and heats to ~2000 K) the total energy's excursion
    falls ~4x when dt is halved (the integrator's O(dt^2)) and stays below
    3e-5 eV/atom at 2 fs (measured 1.1e-5)."""
    pot = _pot(orc, synthetic())
    w = fcc_wire(2.0, 2.0)
    v0 = orc.init_velocities(w.kind, 5, 300.0)
    exc = []
    for dt, n in ((2.0, 500), (1.0, 1000)):
        st = orc.WireState(x=w.x.copy(), v=v0.copy(), kind=w.kind, L0=w.L0)
        e = []
        for _ in range(10):
            orc.md_steps(st, n // 10, dt, pot=pot, brute_max=10**6)
            ob = orc.observables(st, pot=pot)
            e.append(ob.e_pot + ob.e_kin)
        exc.append((max(e) - min(e)) / w.n)
    assert exc[0] < 3e-5
    assert 2.5 < exc[0] / exc[1] < 6.0


def test_tbsma_sampled_trajectory_follows_tbsma(orc):
    """Langevin at 298 K with the pull on, same Philox noise: with the tables
    sampling Eq. 1-2 the EAM trajectory stays within 1e-6 A of TB-SMA's over
    100 steps (the forces differ by the interpolation error, ~1e-6)."""
    w = fcc_wire(2.0, 2.0)
    v0 = orc.init_velocities(w.kind, 7, 298.0)
    out = []
    for pot in (orc.AU, _pot(orc, tbsma_sampled(d_r=0.0005))):
        st = orc.WireState(x=w.x.copy(), v=v0.copy(), kind=w.kind, L0=w.L0, strain_rate=1e9,
                           temperature=298.0, gamma=1e-3, seed=7)
        orc.md_steps(st, 100, 2.0, pot=pot, brute_max=10**6)
        out.append(st.x)
    d = np.max(np.abs(out[0] - out[1]))
    assert 0.0 < d < 1e-6

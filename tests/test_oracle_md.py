"""Pins of the oracle's integrator, thermostat, grips and observables
(Methods "Simulation details", Eq. 4-5) against closed forms and physics."""

import math

import numpy as np
import pytest

from inputs import KIND_GRIP_LEFT, KIND_GRIP_RIGHT, dimer, fcc_wire, jitter


def _state(orc, x, kind=None, **kw):
    kind = np.zeros(x.shape[0], np.uint8) if kind is None else kind
    return orc.WireState(x=x.copy(), v=np.zeros_like(x), kind=kind, L0=kw.pop("L0", 1.0), **kw)


def _dimer_k(P):
    s = math.log(P.p * P.A / (P.q * P.xi)) / (P.p - P.q)
    r = P.r0 * (1 + s)
    k = 2 * P.A * (P.p / P.r0) ** 2 * math.exp(-P.p * s) - 2 * P.xi * (P.q / P.r0) ** 2 * math.exp(-P.q * s)
    return r, k


def test_dimer_vibration_period(orc):
    """Small oscillation of a dimer: period 2 pi sqrt(mu / k), mu = m/2, with
    k = E''(r*) from the closed form.  Pins mass, units and the B/A steps."""
    P = orc.AU
    r_star, k = _dimer_k(P)
    mu = 0.5 * orc.MASS_AU * orc.mvv2e()  # eV fs^2 / A^2
    period = 2 * math.pi * math.sqrt(mu / k)
    st = _state(orc, dimer(r_star + 0.002))
    dt = 0.25
    rs = []
    for _ in range(int(3.2 * period / dt)):
        orc.md_steps(st, 1, dt)
        rs.append(st.x[1, 0] - st.x[0, 0] - r_star)
    rs = np.array(rs)
    # upward zero crossings, linearly interpolated
    idx = np.where((rs[:-1] < 0) & (rs[1:] >= 0))[0]
    t = (idx + rs[idx] / (rs[idx] - rs[idx + 1])) * dt
    measured = np.mean(np.diff(t))
    assert measured == pytest.approx(period, rel=2e-3)


def test_velocity_verlet_energy_error_is_second_order(orc):
    """NVE (gamma = 0): the energy error of velocity Verlet shrinks as dt^2."""
    P = orc.AU
    r_star, _ = _dimer_k(P)
    amp = []
    for dt in (2.0, 1.0):
        st = _state(orc, dimer(r_star + 0.05))
        e0 = orc.energy(st.x)
        es = []
        for _ in range(int(400 / dt)):
            orc.md_steps(st, 1, dt)
            es.append(orc.energy(st.x) + 0.5 * orc.MASS_AU * orc.mvv2e() * np.sum(st.v**2) - e0)
        amp.append(np.max(np.abs(es)))
    assert amp[0] / amp[1] == pytest.approx(4.0, rel=0.1)


def test_nve_wire_energy_conservation(orc):
    """NVE on an unrelaxed wire heating to ~185 K by surface relaxation.  With
    the 5.8 A hard cutoff the total energy jumps each time a pair crosses r_cut,
    whatever dt; with the cutoff moved out to 9 A (where the jumps are ~1e-7 eV)
    the remaining error is velocity Verlet's and falls as dt^2."""
    import dataclasses

    P = dataclasses.replace(orc.AU, r_cut=9.0)
    w = fcc_wire(2.0, 3.0)
    kind = np.zeros(w.n, np.uint8)  # no grips: a free wire
    m = orc.MASS_AU * orc.mvv2e()
    dev = {}
    for dt in (2.0, 1.0):
        st = _state(orc, w.x, kind)
        st.v = orc.init_velocities(kind, seed=3, T=10.0)
        e0 = orc.energy(st.x, P) + 0.5 * m * np.sum(st.v**2)
        d = []
        for _ in range(10):
            orc.md_steps(st, int(100 / dt), dt, pot=P)
            d.append(orc.energy(st.x, P) + 0.5 * m * np.sum(st.v**2) - e0)
        dev[dt] = np.abs(np.array(d)).max() / w.n
        assert abs(np.sum(st.v, axis=0)).max() * m < 1e-9  # momentum (no grips, no noise)
    assert dev[2.0] < 2e-5
    assert dev[2.0] / dev[1.0] == pytest.approx(4.0, rel=0.15)


def _free_atoms(n, spacing=7.0):
    g = int(np.ceil(n ** (1 / 3)))
    idx = np.stack(np.meshgrid(np.arange(g), np.arange(g), np.arange(g), indexing="ij"), -1)
    return spacing * idx.reshape(-1, 3)[:n].astype(np.float64)


def test_free_particle_drift_is_exact(orc):
    x = _free_atoms(64)
    st = _state(orc, x)
    rng = np.random.default_rng(0)
    st.v = rng.standard_normal(x.shape) * 1e-3
    v0 = st.v.copy()
    orc.md_steps(st, 10, 2.0)
    assert np.allclose(st.x, x + 20.0 * v0, rtol=0, atol=1e-13)
    assert np.array_equal(st.v, v0)


def test_ornstein_uhlenbeck_law_of_the_O_step(orc):
    """Free atoms under the O step: after n steps the mean is c1^n v0 and the
    variance (kT/m)(1 - c1^{2n}), c1 = exp(-gamma dt)."""
    x = _free_atoms(1728)
    T, gamma, dt, n = 300.0, 0.01, 2.0, 40
    st = _state(orc, x, temperature=T, gamma=gamma, seed=99)
    u = 0.004
    st.v[:] = u
    orc.md_steps(st, n, dt)
    c1 = math.exp(-gamma * dt)
    sig2 = orc.kb() * T / (orc.MASS_AU * orc.mvv2e())
    var = sig2 * (1 - c1 ** (2 * n))
    samples = st.v.reshape(-1)
    m = samples.size
    assert samples.mean() == pytest.approx(u * c1**n, abs=5 * math.sqrt(var / m))
    assert samples.var() == pytest.approx(var, rel=5 * math.sqrt(2 / m))


def test_thermostat_equipartition(orc):
    """gamma > 0 brings a wire to <T> = T_target (all atoms mobile)."""
    w = fcc_wire(2.0, 2.0)
    kind = np.zeros(w.n, np.uint8)
    st = _state(orc, w.x, kind, temperature=50.0, gamma=0.02, seed=4)
    orc.md_steps(st, 300, 2.0)
    temps = []
    for _ in range(60):
        orc.md_steps(st, 10, 2.0)
        temps.append(orc.observables(st).temp)
    assert np.mean(temps) == pytest.approx(50.0, rel=0.1)


def test_grips_rigid_pull_closed_form(orc):
    w = fcc_wire(2.0, 3.0, strain_rate=1e9)
    st = _state(orc, w.x, w.kind, L0=w.L0, strain_rate=1e9, temperature=10.0, gamma=1e-3)
    st.v = orc.init_velocities(w.kind, 0, 10.0)
    n, dt = 25, 2.0
    orc.md_steps(st, n, dt)
    delta = 1e9 * 1e-15 * w.L0 * dt / 2
    L = w.kind == KIND_GRIP_LEFT
    R = w.kind == KIND_GRIP_RIGHT
    assert np.allclose(st.x[L, 0], w.x[L, 0] - n * delta, atol=1e-12)
    assert np.allclose(st.x[R, 0], w.x[R, 0] + n * delta, atol=1e-12)
    assert np.array_equal(st.x[L | R, 1:], w.x[L | R, 1:])
    assert np.all(st.v[L | R] == 0)
    ob = orc.observables(st)
    # strain of Eq. 4: each end moved n*delta, so eps = 2 n delta / L0 = strain_rate * n * dt
    assert ob.strain == pytest.approx(1e9 * n * dt * 1e-15, rel=1e-12)


def test_initial_velocities(orc):
    w = fcc_wire(2.0, 6.0)
    v = orc.init_velocities(w.kind, seed=12, T=298.0)
    mob = w.kind == 0
    assert np.all(v[~mob] == 0)
    assert np.abs(v[mob].sum(axis=0)).max() < 1e-14
    m = orc.MASS_AU * orc.mvv2e()
    T = m * np.sum(v[mob] ** 2) / (3 * mob.sum() * orc.kb())
    assert T == pytest.approx(298.0, rel=1e-12)
    # same seed, same draw; other seed, other draw
    assert np.array_equal(v, orc.init_velocities(w.kind, seed=12, T=298.0))
    assert not np.array_equal(v, orc.init_velocities(w.kind, seed=13, T=298.0))


def test_virial_stress_is_strain_derivative_of_energy(orc):
    """At T = 0 Eq. 5 reduces to V sigma_xx = sum_i 1/2 sum_j r_x,ij F_x,ij,
    which equals dE/d(eps) under an affine axial stretch x -> (1+eps) x.
    Pins sign (tension positive) and the factor 1/2."""
    w = fcc_wire(2.0, 3.0)
    x = jitter(w.x, 0.03, seed=2)
    st = _state(orc, x, w.kind, L0=w.L0)
    ob = orc.observables(st)
    h = 1e-5

    def e(eps):
        y = x.copy()
        y[:, 0] *= 1 + eps
        return orc.energy(y)

    dE = (-e(2 * h) + 8 * e(h) - 8 * e(-h) + e(-2 * h)) / (12 * h)
    assert ob.virial_xx == pytest.approx(dE, rel=1e-6, abs=1e-6)
    P = orc.AU
    V = w.n * 4 / 3 * math.pi * (P.r0 / 2) ** 3
    assert ob.sigma_xx == pytest.approx(ob.virial_xx / V, rel=1e-12)
    # a stretched perfect wire is in tension
    y = w.x.copy()
    y[:, 0] *= 1.02
    assert orc.observables(_state(orc, y, w.kind, L0=w.L0)).sigma_xx > 0


def test_kinetic_term_of_the_stress(orc):
    x = _free_atoms(27)
    st = _state(orc, x)
    st.v[:, 0] = 0.01
    ob = orc.observables(st)
    m = orc.MASS_AU * orc.mvv2e()
    V = 27 * 4 / 3 * math.pi * (orc.AU.r0 / 2) ** 3
    assert ob.sigma_xx == pytest.approx(-m * 27 * 0.01**2 / V, rel=1e-12)
    assert ob.e_kin == pytest.approx(0.5 * m * 27 * 0.01**2, rel=1e-12)


def test_rebuild_counter(orc):
    w = fcc_wire(2.0, 2.0)
    st = _state(orc, w.x, np.zeros(w.n, np.uint8))
    orc.md_steps(st, 5, 2.0)  # unrelaxed surface atoms move a little
    x = _free_atoms(8)
    st = _state(orc, x)
    st.v[:, 0] = 0.01  # 0.02 A per step; r_skin/2 = 0.145 A -> every 8th step
    orc.md_steps(st, 40, 2.0)
    assert st.n_rebuild == 40 // 8


def test_batch_equals_single_wires(orc):
    wires = [fcc_wire(2.0, 2.0, temperature=10.0, strain_rate=1e9, seed=1),
             fcc_wire(2.0, 3.0, temperature=298.0, strain_rate=1e9, seed=2)]
    from inputs import pack

    b = pack(wires)
    x = b.x.copy()
    v = np.concatenate([orc.init_velocities(w.kind, w.seed, w.temperature) for w in wires])
    x0, v0 = x.copy(), v.copy()
    orc.md_batch(x, v, b.kind, b.offset, b.n, b.L0, b.strain_rate, b.temperature, b.gamma,
                 b.seed, 0, 10, 2.0)
    for w_i, w in enumerate(wires):
        s = b.wire_slice(w_i)
        st = orc.WireState(x=x0[s].copy(), v=v0[s].copy(), kind=w.kind, L0=w.L0,
                           strain_rate=w.strain_rate, temperature=w.temperature, gamma=w.gamma,
                           seed=w.seed)
        orc.md_steps(st, 10, 2.0)
        assert np.array_equal(st.x, x[s]) and np.array_equal(st.v, v[s])

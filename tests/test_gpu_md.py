"""Dynamics checks of the CUDA path on the GPU: NVE energy conservation
(velocity Verlet with gamma = 0; the target is a drift below 1e-4 eV/atom/ns),
the Langevin thermostat's temperature, and the force-error gate (a7) checked
every 1000 steps along a pulled run."""

import numpy as np
import pytest

from inputs import Wire, fcc_wire, pack

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def tb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1311_3890_b300 as tb

    tb.lib()
    return tb


def _relaxed_wire(tb, seed):
    """D2 x L6 wire (1035 atoms) relaxed by strongly damped dynamics at T = 0."""
    w = fcc_wire(2.0, 6.0)
    relax = Wire(x=w.x, kind=w.kind, diameter_nm=2.0, length_nm=6.0, L0=w.L0, temperature=0.0,
                 strain_rate=0.0, gamma=0.02, seed=seed)
    eng = tb.Engine(pack([relax]), precision="fp64")
    eng.step(4000, 2.0)
    x = eng.positions()
    eng.close()
    return w, x


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("T", [10.0, 298.0])
def test_nve_energy_drift(tb, prec, T):
    """Relaxed wire, 20 ps of Langevin at T, then 100 ps of NVE (gamma = 0,
    grips held): the linear drift of E_pot + E_kin per atom stays below
    1e-4 eV/atom/ns.  (Without the equilibration the fit would include the
    equipartition transient, during which pairs crossing the hard 5.8 A
    cutoff change the energy in a biased way.)"""
    w, x = _relaxed_wire(tb, 1)
    eq = Wire(x=x, kind=w.kind, diameter_nm=2.0, length_nm=6.0, L0=w.L0, temperature=T,
              strain_rate=0.0, gamma=0.01, seed=5)
    e_eq = tb.Engine(pack([eq]), precision=prec)
    e_eq.init_velocities()
    e_eq.step(10000, 2.0)
    x_eq, v_eq = e_eq.positions(), e_eq.velocities()
    e_eq.close()
    nve = Wire(x=x_eq, kind=w.kind, diameter_nm=2.0, length_nm=6.0, L0=w.L0, temperature=T,
               strain_rate=0.0, gamma=0.0, seed=5)
    eng = tb.Engine(pack([nve]), precision=prec)
    eng.upload(None, np.ascontiguousarray(v_eq.T).reshape(-1))
    n = w.n
    t_ps, e = [], []
    for k in range(51):  # 100 ps in 2000-step blocks (4 ps)
        if k:
            eng.step(2000, 2.0)
        ob = eng.observables()
        t_ps.append(k * 4.0)
        e.append((ob["e_pot"][0] + ob["e_kin"][0]) / n)
    e = np.array(e)
    slope = np.polyfit(np.array(t_ps) * 1e-3, e, 1)[0]  # eV/atom/ns
    print(f"NVE drift {prec} {T} K: {slope:.3e} eV/atom/ns, std {np.std(e):.2e} eV/atom")
    assert abs(slope) < 1e-4, (prec, T, slope)
    assert np.std(e) < 1e-4  # fluctuation of the total energy per atom
    eng.close()


def test_langevin_temperature(tb):
    w = fcc_wire(2.0, 6.0)
    wire = Wire(x=w.x, kind=w.kind, diameter_nm=2.0, length_nm=6.0, L0=w.L0, temperature=298.0,
                strain_rate=0.0, gamma=0.01, seed=3)
    eng = tb.Engine(pack([wire]), precision="mixed")
    eng.init_velocities()
    eng.step(2000, 2.0)
    temps = []
    for _ in range(40):
        eng.step(100, 2.0)
        temps.append(eng.observables()["temp"][0])
    assert np.mean(temps) == pytest.approx(298.0, rel=0.05)
    eng.close()


def test_force_check_every_1000_steps_along_a_pull(tb):
    """The single D3 x L40 wire (17435 atoms) pulled at 1e8 1/s at 10 K: the
    mixed forces stay within the 1e-5 gate of the FP64 forces at every
    1000-step check."""
    from inputs.configs import workload

    b = workload("wire_d3_l40")
    eng = tb.Engine(b, precision="mixed")
    eng.init_velocities()
    for _ in range(5):
        eng.step(1000, 2.0)
        fc = eng.force_check()
        assert fc["max_err_scaled"][0] <= 1e-5
        assert fc["norm_err"][0] <= 1e-5
    ob = eng.observables()
    assert ob["strain"][0] == pytest.approx(1e8 * 5000 * 2.0 * 1e-15, rel=1e-9)
    eng.close()


@pytest.mark.parametrize("T", [10.0, 298.0])
def test_nve_drift_over_one_ns_mixed(tb, T):
    """The mixed integrator over 1 ns (500k steps) of NVE after 20 ps of
    Langevin at T: its FP64 state takes FP32 increments whose velocity part
    is rounded to nearest (an unbiased rounding; truncation would shrink
    every position increment), and the linear drift of the total energy
    per atom stays below 1e-4 eV/atom/ns."""
    w, x = _relaxed_wire(tb, 2)
    eq = Wire(x=x, kind=w.kind, diameter_nm=2.0, length_nm=6.0, L0=w.L0, temperature=T,
              strain_rate=0.0, gamma=0.01, seed=9)
    e_eq = tb.Engine(pack([eq]), precision="mixed")
    e_eq.init_velocities()
    e_eq.step(10000, 2.0)
    x_eq, v_eq = e_eq.positions(), e_eq.velocities()
    e_eq.close()
    nve = Wire(x=x_eq, kind=w.kind, diameter_nm=2.0, length_nm=6.0, L0=w.L0, temperature=T,
               strain_rate=0.0, gamma=0.0, seed=9)
    eng = tb.Engine(pack([nve]), precision="mixed")
    eng.upload(None, np.ascontiguousarray(v_eq.T).reshape(-1))
    t_ps, e = [], []
    for k in range(101):  # 1 ns in 5000-step blocks (10 ps)
        if k:
            eng.step(5000, 2.0)
        ob = eng.observables()
        t_ps.append(k * 10.0)
        e.append((ob["e_pot"][0] + ob["e_kin"][0]) / w.n)
    e = np.array(e)
    slope = np.polyfit(np.array(t_ps) * 1e-3, e, 1)[0]  # eV/atom/ns
    print(f"NVE drift mixed {T} K over 1 ns: {slope:.3e} eV/atom/ns, std {np.std(e):.2e} eV/atom")
    assert abs(slope) < 1e-4, (T, slope)
    eng.close()

"""Host-side readings of the trajectory observables (yield, failure, neck)
on synthetic report series with known answers."""

import math

import numpy as np
import pytest

from paper_1311_3890_b300.analysis import failure, trailing_mean, yield_point


def test_trailing_mean():
    y = np.array([1.0, 2.0, 3.0, 4.0, 5.0])
    np.testing.assert_allclose(trailing_mean(y, 2), [1.0, 1.5, 2.5, 3.5, 4.5])
    np.testing.assert_allclose(trailing_mean(y, 1), y)
    np.testing.assert_allclose(trailing_mean(y, 10), np.cumsum(y) / np.arange(1, 6))


def test_yield_point_of_a_peaked_curve():
    """Elastic rise, peak at strain 0.05, then softening; noise averaged out
    by the window."""
    eps = np.linspace(0.0, 0.2, 201)
    sigma = np.where(eps < 0.05, 100 * eps, 5.0 - 20 * (eps - 0.05))
    sy, ey = yield_point(eps, sigma, 1)
    assert sy == 5.0 and ey == eps[50]
    noisy = sigma + 0.5 * np.where(np.arange(eps.size) % 2 == 0, 1.0, -1.0)
    sy2, ey2 = yield_point(eps, noisy, 2)
    assert abs(sy2 - 5.0) < 0.2 and abs(ey2 - 0.05) < 0.003


def test_failure_strain_and_final_neck():
    eps = np.arange(10) * 0.1
    conn = np.array([1, 1, 1, 1, 0, 0, 1, 0, 0, 0], dtype=bool)  # first break at report 4
    neck = np.array([30, 28, 20, 9, 0, 0, 3, 0, 0, 0])
    ef, fn = failure(eps, conn, neck)
    assert ef == eps[4] and fn == 9
    ef, fn = failure(eps, np.ones(10, bool), neck)
    assert math.isnan(ef) and fn == -1


def test_critical_length_worked_example():
    """Eq. 6's worked example as printed (golden fixture): D0 = 3.1 nm and
    eps_y = 0.076 give L_C between 40.8 and 57.7 nm."""
    import json
    import os

    from paper_1311_3890_b300.analysis import critical_length

    with open(os.path.join(os.path.dirname(__file__), "golden", "critical_length_eq6.json")) as f:
        g = json.load(f)
    lo, hi = critical_length(g["D0_nm"], g["eps_y"])
    tol = g["printed_precision_nm"]
    assert abs(lo - g["L_C_range_nm_printed"][0]) <= tol
    assert abs(hi - g["L_C_range_nm_printed"][1]) <= tol


def test_observed_critical_length_and_failure_map():
    from paper_1311_3890_b300.analysis import failure_map, observed_critical_length

    # 20 and 40 nm wires fail ductile (post-yield strain 0.3), 60 and 80 nm brittle (0.02)
    L = np.repeat([20.0, 40.0, 60.0, 80.0], 10)
    eps_y = np.full(L.size, 0.08)
    eps_f = eps_y + np.where(L < 50, 0.3, 0.02)
    assert observed_critical_length(L, eps_f, eps_y) == 50.0
    # one brittle outlier among ductile wires does not move it
    eps_f[0] = eps_y[0] + 0.01
    assert observed_critical_length(L, eps_f, eps_y) == 50.0
    h = failure_map(L, eps_f, eps_y, [0, 30, 50, 70, 90], [0.0, 0.1, 1.0])
    np.testing.assert_array_equal(h, [[1, 9], [0, 10], [10, 0], [10, 0]])
    assert np.isnan(observed_critical_length(L[:20], eps_f[:20], eps_y[:20]))


class _FakeEngine:
    """Records the calls paper_protocol makes; grips move by the pull of the
    protocol in force, the wire fails at a fixed grip displacement."""

    def __init__(self, lam, L0=40.0, fail_at=6.0):
        import types

        self.W = 1
        self.batch = types.SimpleNamespace(L0=np.array([L0]))
        self.calls, self.step_count, self.d_grip = [], 100, 0.0
        self.proto, self.lam, self.fail_at = {}, lam, fail_at

    def observables(self):
        L0 = self.batch.L0[0]
        return {"step": np.array([self.step_count]), "strain": np.array([2 * self.d_grip / L0]),
                "sigma_xx": np.array([0.01 * self.d_grip])}

    def set_protocol(self, **kw):
        self.calls.append(("set_protocol", kw))
        self.proto = kw

    def step(self, n, dt):
        self.calls.append(("step", n))
        if self.proto.get("pull") == "stepwise" and self.proto["pull_step"] > 0:
            events = (self.step_count + n) // self.proto["pull_interval"] - \
                self.step_count // self.proto["pull_interval"]
            self.d_grip += events * self.proto["pull_step"]
        self.step_count += n

    def barostat(self):
        return np.array([self.lam]), np.array([0.0])

    def topology(self):
        return {"connected": np.array([self.d_grip < self.fail_at]), "neck": np.array([3])}


def test_paper_protocol_phases_and_strain_reference():
    """Four phases in order: barostat at t_start with the grips held, ramp and
    hold without barostat, then the stepwise pull; the ramp starts where the
    barostat phase ends (counted from the engine's current step), and the
    strains come back relative to the equilibrated length L0 e^lambda."""
    from paper_1311_3890_b300.analysis import paper_protocol

    lam = -0.04
    eng = _FakeEngine(lam)
    run = paper_protocol(eng, barostat_steps=500, ramp_steps=300, hold_steps=200, pull_step=0.05,
                         pull_interval=20, report_every=100, max_pull_steps=20000)
    sets = [kw for name, kw in eng.calls if name == "set_protocol"]
    steps = [n for name, n in eng.calls if name == "step"]
    assert len(sets) == 3 and steps[:2] == [500, 500]
    assert sets[0]["baro_tau_fs"] > 0 and sets[0]["pull_step"] == 0.0
    assert all(s.get("baro_tau_fs", 0.0) == 0.0 for s in sets[1:])
    assert sets[1]["pull_step"] == 0.0 and sets[2]["pull_step"] == 0.05
    assert all(s["ramp_start"] == 100 + 500 and s["ramp_steps"] == 300 and s["t_start"] == 0.01
               for s in sets)
    assert run.log_stretch[0] == lam
    r = run.results[0]
    # failure at a grip displacement of 6 A: strain 2 * 6 / (40 e^lambda)
    assert r.eps_f == pytest.approx(2 * 6.0 / (40.0 * math.exp(lam)), rel=1e-12)
    assert r.strain[-1] == pytest.approx(2 * eng.d_grip / (40.0 * math.exp(lam)), rel=1e-12)


def test_campaign_and_saved_results(tmp_path):
    """campaign on two fake wires of different length: readings per wire,
    the failure map counts both, and save_results writes every history."""
    from paper_1311_3890_b300.analysis import campaign, save_results

    class TwoWires(_FakeEngine):
        def __init__(self):
            super().__init__(-0.03)
            self.W = 2
            self.batch.L0 = np.array([40.0, 80.0])
            self.d = np.zeros(2)

        def observables(self):
            return {"step": np.array([self.step_count] * 2),
                    "strain": 2 * self.d / self.batch.L0,
                    "sigma_xx": 0.01 * self.d * np.exp(-self.d / 2.0)}  # peaks at 2 A

        def step(self, n, dt):
            before = self.d_grip
            super().step(n, dt)
            self.d += self.d_grip - before

        def barostat(self):
            return np.array([-0.03, -0.03]), np.zeros(2)

        def topology(self):
            return {"connected": self.d < np.array([6.0, 4.0]), "neck": np.array([3, 3])}

    eng = TwoWires()
    c = campaign(eng, [4.0, 8.0], barostat_steps=100, ramp_steps=100, hold_steps=100,
                 pull_step=0.05, pull_interval=20, report_every=100, max_pull_steps=20000)
    f = math.exp(0.03)
    assert c.eps_f == pytest.approx([2 * 6.0 / 40.0 * f, 2 * 4.0 / 80.0 * f], rel=1e-9)
    assert c.failure_map.sum() == 2 and c.failure_map.shape == (2, 20)
    assert np.all(c.eps_y < c.eps_f)
    assert np.all(c.log_stretch == -0.03)
    from paper_1311_3890_b300.analysis import paper_protocol  # noqa: F401

    eng2 = TwoWires()
    run = paper_protocol(eng2, barostat_steps=100, ramp_steps=100, hold_steps=100,
                         pull_step=0.05, pull_interval=20, report_every=100,
                         max_pull_steps=20000)
    p = tmp_path / "run.npz"
    save_results(str(p), run.results)
    z = np.load(p)
    assert set(z.files) >= {"w0_strain", "w1_neck", "eps_f", "final_neck"}
    np.testing.assert_array_equal(z["w1_neck"], run.results[1].neck)

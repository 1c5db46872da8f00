"""Host-side readings of the trajectory observables (yield, failure, neck)
on synthetic report series with known answers."""

import math

import numpy as np

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

"""Pins of the oracle's tabulated EAM (the general form of the two-stage
many-body force the paper builds TB-SMA on; Methods, "TB-SMA potential")
against things other than itself: polynomial exactness and the error order
of the interpolant, closed-form dimer and trimer energies and forces, the
straight-line continuation of the embedding, TB-SMA itself (Eq. 1-3) when
the tables sample its functions, finite differences and invariances."""

import math

import numpy as np
import pytest

from inputs import dimer, fcc_wire, jitter, trimer

from tests._eam_tables import R_CUT, synthetic, tbsma_sampled


def _tab(orc, d):
    return orc.EamTables(**d)


# quadratic test functions: the interpolant must reproduce them exactly
def _fq(r):
    return 0.8 * (6.2 - r) ** 2


def _dfq(r):
    return -1.6 * (6.2 - r)


def _pq(r):
    return 0.3 * (r - 3.4) ** 2 - 0.2


def _dpq(r):
    return 0.6 * (r - 3.4)


def _Fq(rho):
    return -0.9 * rho + 0.05 * rho * rho


def _dFq(rho):
    return -0.9 + 0.1 * rho


def _quadratic_tables(orc, rho_max=40.0, d_r=0.05, d_rho=0.25):
    r = np.arange(int(round(6.0 / d_r)) + 1) * d_r
    rho = np.arange(int(round(rho_max / d_rho)) + 1) * d_rho
    return orc.EamTables(F=_Fq(rho), d_rho=d_rho, f=_fq(r), phi=_pq(r), d_r=d_r, r_cut=5.8)


def test_interpolant_is_exact_for_quadratics_and_linear_past_the_ends(orc):
    h = 0.25
    s = np.arange(9) * h
    y = 3.0 - 2.0 * s + 0.7 * s * s
    rng = np.random.default_rng(0)
    t = rng.uniform(0.0, 2.0, 200)
    v, d = orc.eam_interp(y, h, t)
    np.testing.assert_allclose(v, 3.0 - 2.0 * t + 0.7 * t * t, rtol=0, atol=1e-13)
    np.testing.assert_allclose(d, -2.0 + 1.4 * t, rtol=0, atol=1e-12)
    # past the ends: the tangent line at the end sample
    for t0, end in ((-0.3, 0.0), (2.6, 2.0)):
        v, d = orc.eam_interp(y, h, t0)
        y_e, m_e = 3.0 - 2.0 * end + 0.7 * end * end, -2.0 + 1.4 * end
        assert v[0] == pytest.approx(y_e + m_e * (t0 - end), abs=1e-13)
        assert d[0] == pytest.approx(m_e, abs=1e-12)


def test_interpolant_error_is_third_order(orc):
    """Cubic Hermite with second-order node slopes: the value error falls
    8x per halving of h (a dropped or mis-weighted basis term would show as
    first or second order), the derivative error 4x."""
    errs, derrs = [], []
    t = np.linspace(0.3, 2.7, 997)  # inside: the end intervals use one-sided slopes
    for h in (0.05, 0.025, 0.0125):
        s = np.arange(int(round(3.0 / h)) + 1) * h
        v, d = orc.eam_interp(np.sin(2.0 * s), h, t)
        errs.append(np.max(np.abs(v - np.sin(2.0 * t))))
        derrs.append(np.max(np.abs(d - 2.0 * np.cos(2.0 * t))))
    for a, b in zip(errs, errs[1:]):
        assert 6.0 < a / b < 10.0
    for a, b in zip(derrs, derrs[1:]):
        assert 3.0 < a / b < 5.0


@pytest.mark.parametrize("r", [2.3, 2.884, 3.61, 4.9, 5.79])
def test_dimer_closed_form(orc, r):
    """Two atoms: rho = f(r) each, E = 2 F(f(r)) + phi(r), and
    F_0 = +dE/dr along the axis towards atom 1."""
    tab = _quadratic_tables(orc)
    out = orc.eam(dimer(r), tab)
    rho = _fq(r)
    assert out.E == pytest.approx(2 * _Fq(rho) + _pq(r), rel=1e-13, abs=1e-13)
    dEdr = 2 * _dFq(rho) * _dfq(r) + _dpq(r)
    assert out.F[0, 0] == pytest.approx(dEdr, rel=1e-12, abs=1e-12)
    assert out.F[1, 0] == pytest.approx(-dEdr, rel=1e-12, abs=1e-12)
    assert np.all(out.F[:, 1:] == 0.0)
    np.testing.assert_allclose(out.eR, 0.5 * _pq(r), rtol=1e-13)
    np.testing.assert_allclose(out.eB, _Fq(rho), rtol=1e-13)


def test_dimer_beyond_cutoff_and_tie(orc):
    tab = _quadratic_tables(orc)
    assert orc.eam(dimer(5.8001), tab).E == 2 * _Fq(0.0)
    # r = r_cut interacts
    assert orc.eam(dimer(5.8), tab).E == pytest.approx(2 * _Fq(_fq(5.8)) + _pq(5.8), rel=1e-13)


def _trimer_energy(x):
    rho = np.zeros(3)
    E = 0.0
    for i in range(3):
        for j in range(3):
            if i != j:
                r = np.linalg.norm(x[i] - x[j])
                rho[i] += _fq(r)
                E += 0.5 * _pq(r)
    return E + sum(_Fq(p) for p in rho)


def test_trimer_closed_form_and_forces(orc):
    """A scalene triangle: energy from the closed-form functions, forces by
    central differences of that closed form (a wrong sign, a missing
    F'(rho_j) term or a transposed index fails)."""
    x = trimer(2.9)
    x[2] += np.array([0.31, -0.17, 0.4])
    tab = _quadratic_tables(orc)
    out = orc.eam(x, tab)
    assert out.E == pytest.approx(_trimer_energy(x), rel=1e-13)
    h = 1e-5
    for i in range(3):
        for k in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, k] += h
            xm[i, k] -= h
            g = (_trimer_energy(xp) - _trimer_energy(xm)) / (2 * h)
            assert out.F[i, k] == pytest.approx(-g, rel=1e-8, abs=1e-9)


def test_embedding_continues_linearly_past_the_table(orc):
    """rho beyond the F table's last sample: F = F_end + F'_end (rho - rho_end)."""
    tab = _quadratic_tables(orc, rho_max=10.0)
    r = 2.5  # f(2.5) = 10.95 > 10
    rho = _fq(r)
    out = orc.eam(dimer(r), tab)
    F_lin = _Fq(10.0) + _dFq(10.0) * (rho - 10.0)
    assert out.E == pytest.approx(2 * F_lin + _pq(r), rel=1e-13)
    assert out.F[0, 0] == pytest.approx(2 * _dFq(10.0) * _dfq(r) + _dpq(r), rel=1e-12)


def test_tbsma_sampled_tables_reproduce_tbsma(orc):
    """With f, phi and F sampled from Eq. 1-2 the EAM is TB-SMA up to the
    interpolation error (O(h^3) in the values, O(h^2) in the forces): a
    thermal D2 wire's energy within 1e-8 relative and, with r sampled every
    0.0005 A, every force within 2e-6 of the largest; the force error falls
    3-8x (about 4x) when the r grid is refined 2x."""
    w = fcc_wire(2.0, 3.0)
    x = jitter(w.x, 0.08, 3)
    ref = orc.tbsma(x)
    coarse = orc.eam(x, _tab(orc, tbsma_sampled(d_r=0.001)))
    out = orc.eam(x, _tab(orc, tbsma_sampled(d_r=0.0005)))
    ratio = np.max(np.abs(coarse.F - ref.F)) / np.max(np.abs(out.F - ref.F))
    assert 3.0 < ratio < 8.0  # second order (a first-order slip gives ~2)
    assert out.n_pairs == ref.n_pairs
    assert out.E == pytest.approx(ref.E, rel=1e-8)
    scale = np.max(np.abs(ref.F))
    assert np.max(np.abs(out.F - ref.F)) < 2e-6 * scale
    np.testing.assert_allclose(out.rho, ref.rho, rtol=1e-8)
    np.testing.assert_allclose(out.eR, ref.eR, rtol=1e-7)
    np.testing.assert_allclose(out.w, ref.w, rtol=0, atol=2e-6 * np.max(np.abs(ref.w)))


@pytest.mark.parametrize("which", ["tbsma_sampled", "synthetic"])
def test_forces_are_minus_the_energy_gradient(orc, which):
    tab = _tab(orc, tbsma_sampled() if which == "tbsma_sampled" else synthetic())
    # the first jitter seed with no pair within 1e-3 A of the hard cutoff, so
    # that the differences see no jump
    for seed in range(5, 100):
        x = jitter(fcc_wire(2.0, 1.5).x[:60], 0.1, seed)
        d = np.linalg.norm(x[:, None] - x[None], axis=-1)
        if np.min(np.abs(d - R_CUT)) > 1e-3:
            break
    else:
        pytest.fail("no jitter seed keeps the pairs away from r_cut")
    F = orc.eam(x, tab).F
    h = 1e-5
    rng = np.random.default_rng(1)
    for i in rng.choice(len(x), 12, replace=False):
        for k in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, k] += h
            xm[i, k] -= h
            g = (orc.eam_energy(xp, tab) - orc.eam_energy(xm, tab)) / (2 * h)
            assert F[i, k] == pytest.approx(-g, rel=1e-6, abs=1e-7)


def test_net_force_zero_and_rotation_covariance(orc):
    x = jitter(fcc_wire(2.0, 3.0).x, 0.1, 7)
    tab = _tab(orc, synthetic())
    out = orc.eam(x, tab)
    assert np.max(np.abs(out.F.sum(axis=0))) < 1e-10
    th = 0.7
    R = np.array([[1, 0, 0], [0, math.cos(th), -math.sin(th)], [0, math.sin(th), math.cos(th)]])
    rot = orc.eam(x @ R.T + np.array([3.0, -1.0, 2.0]), tab)
    assert rot.E == pytest.approx(out.E, rel=1e-12)
    np.testing.assert_allclose(rot.F, out.F @ R.T, rtol=0, atol=1e-10)


def test_cells_and_brute_force_agree(orc):
    x = jitter(fcc_wire(2.0, 3.0).x, 0.1, 9)
    tab = _tab(orc, synthetic())
    a = orc.eam(x, tab, brute_max=10**6)
    b = orc.eam(x, tab, brute_max=0)
    assert a.n_pairs == b.n_pairs
    np.testing.assert_array_equal(a.F, b.F)

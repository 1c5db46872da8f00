"""The library's EAM table construction on the host (tbsma_eam_cubics, the
coefficients tbsma_set_eam uploads; no GPU) against the oracle's
interpolant: same values and slopes at the nodes, inside the intervals and
for sample tables that are not smooth."""

import numpy as np
import pytest

from tests._eam_tables import synthetic, tbsma_sampled


def _eval(c, h, s):
    k = np.minimum((s / h).astype(np.int64), len(c) - 1)
    t = s / h - k
    a = c[k]
    v = a[:, 0] + t * (a[:, 1] + t * (a[:, 2] + t * a[:, 3]))
    d = (a[:, 1] + t * (2 * a[:, 2] + 3 * a[:, 3] * t)) / h
    return v, d


@pytest.fixture(scope="module")
def tb():
    import paper_1311_3890_b300 as tb

    tb.lib()  # the library loads without a GPU; this entry needs none
    return tb


@pytest.mark.parametrize("name", ["f", "phi", "F"])
@pytest.mark.parametrize("which", ["tbsma_sampled", "synthetic"])
def test_cubics_equal_the_oracle_interpolant(tb, orc, which, name):
    T = (tbsma_sampled if which == "tbsma_sampled" else synthetic)()
    y = T[name]
    h = T["d_rho"] if name == "F" else T["d_r"]
    c = tb.eam_cubics(y)
    assert c.shape == (y.size - 1, 4)
    rng = np.random.default_rng(3)
    s = np.concatenate([np.arange(y.size - 1) * h, rng.uniform(0, (y.size - 1) * h, 4000)])
    v, d = _eval(c, h, s)
    vo, do = orc.eam_interp(y, h, s)
    scale = np.max(np.abs(y))
    np.testing.assert_allclose(v, vo, rtol=0, atol=1e-13 * scale)
    dscale = np.max(np.abs(do))
    np.testing.assert_allclose(d, do, rtol=0, atol=1e-11 * dscale)
    # at the nodes the cubic takes the samples exactly
    np.testing.assert_array_equal(c[:, 0], y[:-1])


def test_cubics_of_rough_samples(tb, orc):
    y = np.random.default_rng(4).normal(size=50)
    c = tb.eam_cubics(y)
    s = np.linspace(0.0, 49 * 0.1, 3001)
    v, d = _eval(c, 0.1, s)
    vo, do = orc.eam_interp(y, 0.1, s)
    np.testing.assert_allclose(v, vo, rtol=0, atol=1e-13)
    np.testing.assert_allclose(d, do, rtol=0, atol=1e-11)


def test_cubics_reject_short_tables(tb):
    with pytest.raises(tb.TbsmaError):
        tb.eam_cubics(np.zeros(2))

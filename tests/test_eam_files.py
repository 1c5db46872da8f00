"""setfl reading (host logic): tables written from analytic functions come
back sample for sample, for one and for two elements, and feed the
oracle's EAM to the same forces as the original tables."""

import numpy as np
import pytest

from inputs import fcc_wire, jitter
from paper_1311_3890_b300.eam_files import read_setfl, write_setfl
from tests._eam_tables import synthetic


def _elem(name, z, T, scale=1.0):
    return dict(name=name, z=z, mass=196.966569, lattice=4.079, kind="fcc", F=scale * T["F"],
                f=scale * T["f"])


def test_one_element_round_trip(tmp_path, orc):
    T = synthetic()
    n_r, n_rho = T["f"].size, T["F"].size
    r = np.arange(n_r) * T["d_r"]
    path = str(tmp_path / "au.setfl")
    write_setfl(path, [_elem("Au", 79, T)], {(0, 0): r * T["phi"]}, n_rho, T["d_rho"], n_r,
                T["d_r"], T["r_cut"], comments=("synthetic Au-like EAM", "", ""))
    got = read_setfl(path)
    assert got["element"] == "Au" and got["d_r"] == T["d_r"] and got["r_cut"] == T["r_cut"]
    np.testing.assert_array_equal(got["F"], T["F"])
    np.testing.assert_array_equal(got["f"], T["f"])
    np.testing.assert_allclose(got["phi"][1:], T["phi"][1:], rtol=1e-15)
    # phi(0) continued by the quadratic through samples 1-3
    assert got["phi"][0] == pytest.approx(3 * T["phi"][1] - 3 * T["phi"][2] + T["phi"][3], rel=1e-14)
    x = jitter(fcc_wire(2.0, 2.0).x, 0.05, 1)
    keys = ("F", "d_rho", "f", "phi", "d_r", "r_cut")
    a = orc.eam(x, orc.EamTables(**{k: T[k] for k in keys}))
    b = orc.eam(x, orc.EamTables(**{k: got[k] for k in keys}))
    np.testing.assert_allclose(b.F, a.F, rtol=0, atol=1e-12)


def test_second_element_of_two(tmp_path):
    T = synthetic()
    n_r, n_rho = T["f"].size, T["F"].size
    r = np.arange(n_r) * T["d_r"]
    pairs = {(0, 0): r * T["phi"], (1, 0): 0.5 * r * T["phi"], (1, 1): 2.0 * r * T["phi"]}
    path = str(tmp_path / "two.setfl")
    write_setfl(path, [_elem("Ag", 47, T), _elem("Au", 79, T, 1.5)], pairs, n_rho, T["d_rho"], n_r,
                T["d_r"], T["r_cut"])
    got = read_setfl(path, "Au")
    assert got["element"] == "Au"
    np.testing.assert_allclose(got["F"], 1.5 * T["F"], rtol=1e-15)
    np.testing.assert_allclose(got["phi"][1:], 2.0 * T["phi"][1:], rtol=1e-15)
    assert read_setfl(path, 1)["element"] == "Au"


def test_truncated_file_is_rejected(tmp_path):
    T = synthetic()
    path = str(tmp_path / "cut.setfl")
    n_r = T["f"].size
    write_setfl(path, [_elem("Au", 79, T)], {(0, 0): np.arange(n_r) * T["d_r"] * T["phi"]},
                T["F"].size, T["d_rho"], n_r, T["d_r"], T["r_cut"])
    lines = open(path).read().splitlines()
    with open(path, "w") as fh:
        fh.write("\n".join(lines[:-20]) + "\n")
    with pytest.raises(ValueError):
        read_setfl(path)
    with pytest.raises(ValueError):
        read_setfl(path, "Cu")

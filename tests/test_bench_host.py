"""Host-side arithmetic of bench.py (no GPU): the timed call sequence, the
kernel count it claims, and the force pass's roofline numbers."""

import math

import pytest

import bench


def test_chunks_report_every_1000_steps():
    assert bench._chunks(10000) == [1000] * 10
    assert bench._chunks(2500) == [1000, 1000, 500]
    assert bench._chunks(30) == [30]


def test_launch_count_of_the_default_run():
    """10000 steps: 200 graph replays of 50 steps (4 kernels per step plus the
    closing half kick each), 10 reports of 5 kernels, and the rebuild chains
    the library counted (one per step and per report's refresh: 4 kernels
    each): the 80290 of the bench line."""
    chains = 10000 + 10
    assert bench.launches_in(10000, chains) == 200 * (4 * 50 + 1) + 10 * 5 + 4 * chains == 80290
    # a call shorter than the graph is captured whole: one closing kernel
    assert bench.launches_in(30, 30) == 4 * 30 + 1 + 5 + 4 * 30


def test_roofline_bound_and_fraction():
    """The bench workload's census (44.87 in-cutoff and 0.82 skin entries per
    atom): FP32-bound; the roofline time is the FP32 work at 128 lanes per
    SM and clock, and the fraction is that time over the measured one."""
    N, n_c, n_s, sms, mhz = 4463360, 44.87, 0.82, 148, 2032.0
    r = bench.roofline_of(N, n_c, n_s, 0.2747, sms, mhz, 6503.7)
    t_fp32 = N * (21 * n_c + 7 * n_s) / (128 * sms * mhz * 1e6)
    assert r["bound"] == "alu" and r["unit"] == "T FP32-inst/s"
    assert math.isclose(r["roofline_ms"], 1e3 * t_fp32, rel_tol=1e-12)
    assert math.isclose(r["frac"], r["roofline_ms"] / 0.2747, rel_tol=1e-12)
    assert 0.39 < r["frac"] < 0.41
    assert r["t_mufu_ms"] < r["t_fp32_ms"] and r["t_hbm_ms"] < r["t_fp32_ms"]
    # the same work on a slow memory is HBM-bound
    h = bench.roofline_of(N, n_c, n_s, 0.2747, sms, mhz, 1000.0)
    assert h["bound"] == "hbm" and h["unit"] == "GB/s"
    assert math.isclose(h["frac"], h["hbm_frac"], rel_tol=1e-12)


def test_eam_roofline_and_tables():
    """--potential eam: 25 FP32 instructions and one MUFU op per in-cutoff
    entry; the Au tables cover r_cut and sample the TB-SMA functions."""
    N, n_c, n_s, sms, mhz = 4463360, 44.87, 0.82, 148, 2032.0
    r = bench.roofline_of(N, n_c, n_s, 0.30, sms, mhz, 6503.7, per_in=bench.EAM_PER_IN)
    assert r["bound"] == "alu" and r["unit"] == "T FP32-inst/s"
    assert math.isclose(r["roofline_ms"], 1e3 * N * (25 * n_c + 7 * n_s) / (128 * sms * mhz * 1e6),
                        rel_tol=1e-12)
    t = bench.au_eam_tables()
    assert (t["f"].size - 1) * t["d_r"] >= 5.8 and t["f"].size == t["phi"].size
    k = int(round(2.884 / t["d_r"]))
    assert math.isclose(t["f"][k], 1.790 ** 2 * math.exp(-2 * 4.036 * (k * t["d_r"] / 2.884 - 1)))
    assert t["F"][0] == 0.0 and math.isclose(t["F"][-1], -math.sqrt((t["F"].size - 1) * t["d_rho"]))


def test_oracle_sample_runs_the_eam(orc):
    """The cpu_baseline leg of --potential eam times the oracle's EAM MD."""
    from inputs import workload

    b = workload("tiny_batch")
    v, cores, desc, n, steps = bench.oracle_sample(b, budget_s=0.1, steps=2, eam=True)
    assert v > 0 and steps == 2 and "EAM" in desc and n == b.n[:cores].sum()


def test_workload_atoms_matches_the_built_batch():
    from inputs.configs import WORKLOADS, build

    for name in ("tiny_batch", "paper_table2"):
        specs = WORKLOADS[name]()
        assert bench._workload_atoms(specs) == build(specs).n_atoms


@pytest.mark.parametrize("k,atoms", [(1, 8939), (12, 106289)])
def test_table2_wires_are_close_to_the_papers(k, atoms):
    """The Table 2 wires (D3.1 x L20.4k nm) come out within 1.5 % of the
    paper's atom counts (8823 ... 106173)."""
    from inputs.configs import WORKLOADS

    spec = WORKLOADS["paper_table2"]()[k - 1]
    assert bench._workload_atoms([spec]) == atoms
    assert abs(atoms / bench.TABLE2_ATOMS[k - 1] - 1.0) < 0.015

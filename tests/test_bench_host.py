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
    closing half kick each), 10 reports folded into the calls' last steps
    (the reduce kernel each), and the rebuild chains the library counted
    (one per step: 7 kernels each, the two envelope passes, the four of the
    cell build and the slab build)."""
    chains = 10000
    assert bench.launches_in(10000, chains) == 200 * (4 * 50 + 1) + 10 * 1 + 7 * chains == 110210
    # a call shorter than the graph is captured whole: one closing kernel
    assert bench.launches_in(30, 30) == 4 * 30 + 1 + 1 + 7 * 30


def test_launch_count_in_the_persistent_step_kernel():
    """50000 steps of a small context: 50 calls of 1000 steps, each one
    launch of the persistent kernel, and 50 reports of 5 kernels plus a
    rebuild chain of 7 (the per-step plans inside the kernel launch
    nothing)."""
    assert bench.launches_in(50000, 50000 + 50, persistent=True) == 50 * (1 + 5 + 7) == 650
    assert bench.launches_in(30, 31, persistent=True) == 1 + 5 + 7


def test_roofline_bound_and_fraction():
    """A census of 44.87 in-cutoff and 0.82 skin entries per atom: the force
    pass is FP32-bound on the method's count (19 FP32 + 3 MUFU per in-cutoff
    pair); the roofline time is that FP32 work at 128 lanes per SM and
    clock, and the fraction is that time over the measured one."""
    N, n_c, n_s, sms, mhz = 4463360, 44.87, 0.82, 148, 2032.0
    r = bench.roofline_of(N, n_c, n_s, 0.2747, sms, mhz, 6503.7)
    t_fp32 = N * 19 * n_c / (128 * sms * mhz * 1e6)
    assert r["bound"] == "alu" and r["unit"] == "T FP32-inst/s"
    assert math.isclose(r["roofline_ms"], 1e3 * t_fp32, rel_tol=1e-12)
    assert math.isclose(r["frac"], r["roofline_ms"] / 0.2747, rel_tol=1e-12)
    assert 0.34 < r["frac"] < 0.36
    assert r["t_mufu_ms"] < r["t_fp32_ms"] and r["t_hbm_ms"] < r["t_fp32_ms"]
    # this implementation's count (conversions and skin entries included)
    i = bench.roofline_of(N, n_c, n_s, 0.2747, sms, mhz, 6503.7, model=bench.FORCE_IMPL_MODEL)
    assert math.isclose(i["roofline_ms"], 1e3 * N * (21 * n_c + 7 * n_s) / (128 * sms * mhz * 1e6),
                        rel_tol=1e-12)
    # the density pass: 11 FP32 + 2 MUFU per pair
    d = bench.roofline_of(N, n_c, n_s, 0.2288, sms, mhz, 6503.7, model=bench.PASS_MODEL["density"])
    assert math.isclose(d["t_fp32_ms"], 1e3 * N * 11 * n_c / (128 * sms * mhz * 1e6), rel_tol=1e-12)
    assert math.isclose(d["t_mufu_ms"], 1e3 * N * 2 * n_c / (32 * sms * mhz * 1e6), rel_tol=1e-12)
    # the same work on a slow memory is HBM-bound
    h = bench.roofline_of(N, n_c, n_s, 0.2747, sms, mhz, 1000.0)
    assert h["bound"] == "hbm" and h["unit"] == "GB/s"
    assert math.isclose(h["frac"], h["hbm_frac"], rel_tol=1e-12)


def test_eam_roofline_and_tables():
    """--potential eam: 25 FP32 instructions and one MUFU op per in-cutoff
    entry; the Au tables cover r_cut and sample the TB-SMA functions."""
    N, n_c, n_s, sms, mhz = 4463360, 44.87, 0.82, 148, 2032.0
    r = bench.roofline_of(N, n_c, n_s, 0.30, sms, mhz, 6503.7, model=bench.EAM_MODEL)
    assert r["bound"] == "alu" and r["unit"] == "T FP32-inst/s"
    assert math.isclose(r["roofline_ms"], 1e3 * N * (25 * n_c + 7 * n_s) / (128 * sms * mhz * 1e6),
                        rel_tol=1e-12)
    t = bench.au_eam_tables()
    assert (t["f"].size - 1) * t["d_r"] >= 5.8 and t["f"].size == t["phi"].size
    k = int(round(2.884 / t["d_r"]))
    assert math.isclose(t["f"][k], 1.790 ** 2 * math.exp(-2 * 4.036 * (k * t["d_r"] / 2.884 - 1)))
    assert t["F"][0] == 0.0 and math.isclose(t["F"][-1], -math.sqrt((t["F"].size - 1) * t["d_rho"]))


def test_stratified_sample_covers_every_stratum():
    """The sweep's comparison legs sample every (diameter, temperature)
    stratum, spread over its lengths, largest wires first."""
    from inputs.configs import WORKLOADS

    specs = WORKLOADS["sweep2048"]()
    atoms = bench._spec_atoms(specs)
    st = bench.strata_of(specs)
    assert len(st) == 6 and sum(len(v) for v in st.values()) == 2048
    picks = bench.stratified_sample(specs, atoms, 2)
    assert len(picks) == 12 and len(set(picks)) == 12
    assert {(specs[w].diameter_nm, specs[w].temperature) for w in picks} == set(st)
    assert [atoms[w] for w in picks] == sorted((atoms[w] for w in picks), reverse=True)
    for key, ws in st.items():  # two different lengths per stratum
        got = [w for w in picks if w in ws]
        assert len({specs[w].length_nm for w in got}) == 2


def test_extrapolation_weights_strata_by_atoms():
    """Per-stratum rates combine as a harmonic mean weighted by atoms: a
    stratum at half the rate with the same atoms gives 2/3 of the fast rate."""
    from inputs.configs import WireSpec

    specs = [WireSpec(2.0, 10.0, 10.0, 1e8, 0), WireSpec(2.0, 10.0, 298.0, 1e8, 1)]
    atoms = [1000, 1000]
    rate = bench.extrapolate(specs, atoms, {0: (2000.0, 1.0), 1: (1000.0, 1.0)})
    assert math.isclose(rate, 2000.0 * 2 / 3, rel_tol=1e-12)


def test_oracle_sample_runs_the_eam(orc):
    """The cpu_baseline leg of --potential eam times the oracle's EAM MD."""
    from inputs import workload

    b = workload("tiny_batch")
    v, cores, desc, n, steps = bench.oracle_sample(b, budget_s=0.1, steps=2, eam=True)
    assert v > 0 and steps == 2 and "EAM" in desc and n == b.n[:b.n_wires].sum()
    v, cores, desc, n, steps = bench.oracle_sample(b, budget_s=0.1, steps=2, wires=[2, 0])
    assert v > 0 and n == b.n[0] + b.n[2]


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

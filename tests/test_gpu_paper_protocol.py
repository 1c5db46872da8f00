"""The paper's whole protocol on the GPU (analysis.paper_protocol: barostat
at 0.01 K, temperature ramp, hold, stepwise elongation to rupture; Methods,
"Simulation details"), with its phases shortened so that the test runs in
seconds."""

import math

import numpy as np
import pytest

from inputs import fcc_wire, pack

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_paper_protocol_equilibrates_and_pulls_to_rupture():
    """Two notched D2 x L4 wires at 10 K: 1500 barostat steps shorten them
    (surface stress: the relaxed 2 nm wire is ~3-4 % shorter), 500 ramp and
    500 hold steps bring them to 10 K, and 0.05 A grip steps every 20 steps
    pull them apart.  The failure strains, measured against the equilibrated
    length, are those of a pulled wire, and the grips moved in whole 0.05 A
    steps."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1311_3890_b300 as tb
    from paper_1311_3890_b300.analysis import paper_protocol

    wires = [fcc_wire(2.0, 4.0, notch_depth=2.5, temperature=10.0, strain_rate=0.0, seed=s)
             for s in range(2)]
    eng = tb.Engine(pack(wires), precision="mixed")
    eng.init_velocities()
    run = paper_protocol(eng, barostat_steps=1500, ramp_steps=500, hold_steps=500,
                         pull_step=0.05, pull_interval=20, report_every=100,
                         max_pull_steps=40000, tau_fs=200.0, baro_tau_fs=100.0)
    assert np.all((run.log_stretch > -0.07) & (run.log_stretch < -0.01))
    for r, w, lam in zip(run.results, wires, run.log_stretch):
        assert math.isfinite(r.eps_f) and 0.05 < r.eps_f < 1.4
        assert r.eps_y < r.eps_f and r.sigma_y > 0
        d_grip = r.strain[-1] * w.L0 * math.exp(lam) / 2.0
        assert d_grip / 0.05 == pytest.approx(round(d_grip / 0.05), abs=1e-6)
    eng.close()


def test_campaign_over_two_lengths(tmp_path):
    """analysis.campaign on notched D2 wires of 4 and 6 nm (shortened
    phases): every wire fails, the failure map counts each wire once in its
    length bin, and the saved histories load back."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1311_3890_b300 as tb
    from paper_1311_3890_b300.analysis import campaign, save_results

    lengths = [4.0, 6.0]
    wires = [fcc_wire(2.0, L, notch_depth=2.5, temperature=10.0, strain_rate=0.0, seed=7)
             for L in lengths]
    eng = tb.Engine(pack(wires), precision="mixed")
    eng.init_velocities()
    c = campaign(eng, lengths, barostat_steps=1000, ramp_steps=300, hold_steps=300,
                 pull_step=0.05, pull_interval=20, report_every=100, max_pull_steps=60000,
                 tau_fs=200.0, baro_tau_fs=100.0)
    assert np.all(np.isfinite(c.eps_f)) and np.all(c.eps_y < c.eps_f)
    assert c.failure_map.sum(axis=1).tolist() == [1, 1]
    eng.close()

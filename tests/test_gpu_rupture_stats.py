"""Rupture statistics, GPU against the oracle (trajectory observables over
many seeds: a single pulled trajectory is chaotic, so beyond short horizons
only the distributions can be compared).

24 notched D2 x L4 wires (580 atoms) at 10 K pulled at 2e10 1/s, Langevin
thermostat, seeds 0..23 on both sides, reports every 100 steps: the failure
strains and yield stresses of the GPU (mixed precision) and of the FP64
oracle must be compatible under a two-sample Kolmogorov-Smirnov test, and
their means close.  Takes about a minute of host time for the oracle.
"""

import numpy as np
import pytest

from inputs import fcc_wire, pack

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")

N_SEEDS = 24
REPORT = 100
MAX_STEPS = 20000


def _wires():
    return [fcc_wire(2.0, 4.0, notch_depth=2.5, temperature=10.0, strain_rate=2e10, seed=s)
            for s in range(N_SEEDS)]


def _oracle_pull(orc, wires):
    """The oracle's Langevin MD on all wires (one per host thread), with the
    oracle's topology and observables at every report."""
    from paper_1311_3890_b300.analysis import failure, yield_point

    b = pack(wires)
    N = b.n_atoms
    x = b.x.copy()
    v = np.zeros_like(x)
    for w in range(b.n_wires):
        s = b.wire_slice(w)
        v[s] = orc.init_velocities(b.kind[s], int(b.seed[w]), float(b.temperature[w]))
    args = (b.kind, b.offset, b.n, b.L0, b.strain_rate, b.temperature, b.gamma, b.seed)
    F = xb = dg = nr = None
    strain, sigma, conn, neck = [], [], [], []
    for k in range(MAX_STEPS // REPORT):
        F, xb, dg, nr = orc.md_batch(x, v, *args, k * REPORT, REPORT, 2.0, brute_max=0, F=F,
                                     x_build=xb, d_grip=dg, n_rebuild=nr)
        row = []
        for w in range(b.n_wires):
            s = b.wire_slice(w)
            st = orc.WireState(x=x[s], v=v[s], kind=b.kind[s], L0=float(b.L0[w]),
                               d_grip=float(dg[w]))
            o = orc.observables(st, brute_max=0)
            t = orc.topology(x[s], b.kind[s])
            row.append((o.strain, o.sigma_xx, t.connected, t.neck))
        row = np.array(row)
        strain.append(row[:, 0])
        sigma.append(row[:, 1])
        conn.append(row[:, 2].astype(bool))
        neck.append(row[:, 3])
        if not np.any(row[:, 2]):
            break
    strain, sigma, conn, neck = map(np.array, (strain, sigma, conn, neck))
    window = max(1, int(round(500.0 / (REPORT * 2.0))))
    ef = np.array([failure(strain[:, w], conn[:, w], neck[:, w])[0] for w in range(b.n_wires)])
    sy = np.array([yield_point(strain[:, w], sigma[:, w], window)[0] for w in range(b.n_wires)])
    return ef, sy


def test_rupture_and_yield_distributions_match_oracle(orc):
    from scipy.stats import ks_2samp

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1311_3890_b300 as tb
    from paper_1311_3890_b300.analysis import pull_to_rupture

    wires = _wires()
    eng = tb.Engine(pack(wires), precision="mixed")
    eng.init_velocities()
    res = pull_to_rupture(eng, report_every=REPORT, max_steps=MAX_STEPS, past_failure=0.0)
    eng.close()
    ef_gpu = np.array([r.eps_f for r in res])
    sy_gpu = np.array([r.sigma_y for r in res])
    ef_ora, sy_ora = _oracle_pull(orc, wires)
    assert np.all(np.isfinite(ef_gpu)) and np.all(np.isfinite(ef_ora))
    print(f"eps_f GPU {ef_gpu.mean():.4f} +- {ef_gpu.std():.4f}, oracle "
          f"{ef_ora.mean():.4f} +- {ef_ora.std():.4f}; sigma_y GPU {sy_gpu.mean():.5f}, "
          f"oracle {sy_ora.mean():.5f} eV/A^3")
    assert ks_2samp(ef_gpu, ef_ora).pvalue > 0.01
    assert ks_2samp(sy_gpu, sy_ora).pvalue > 0.01
    assert abs(ef_gpu.mean() - ef_ora.mean()) < 3 * np.hypot(ef_gpu.std(), ef_ora.std()) / np.sqrt(
        N_SEEDS) + 0.01

"""Tabulated EAM on the GPU (tbsma_set_eam: the general form of the
two-stage many-body force the paper builds TB-SMA on; Methods, "TB-SMA
potential") against the oracle's EAM, through the C ABI.

Tolerances as for TB-SMA (tests/test_gpu_parity.py): FP64 per-atom
|dF_i| <= 1e-12 |F_i| (or 1e-12 S_i for near-zero forces); MIXED per-atom
|dF_i| / S_i <= 1e-5 and ||dF|| / ||F|| <= 1e-5.  The table cubics carry
the same rounding as the exponentials they replace: FP64 coefficients are
formed from sample differences (~1e-15 relative), FP32 ones are rounded
once (6e-8), and the interval coordinate t comes from r with one rounding.
"""

import numpy as np
import pytest

from inputs import jitter, workload
from tests._eam_tables import synthetic, tbsma_sampled
from tests._parity import ambiguous_atoms, force_errors

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TABLES = {"tbsma_sampled": tbsma_sampled, "synthetic": synthetic}


@pytest.fixture(scope="module")
def tb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1311_3890_b300 as tb

    tb.lib()
    return tb


def _batch(sigma, seed):
    b = workload("tiny_batch")
    b.x = jitter(b.x, sigma, seed)
    return b


def _check_fp64(F, ref, amb):
    d, fm, _ = force_errors(F, ref.F)
    ok = np.ones(F.shape[0], bool)
    ok[amb] = False
    big = ok & (fm >= 1e-6 * ref.S)
    assert np.all(d[big] <= 1e-12 * fm[big])
    assert np.all(d[ok & ~big] <= 1e-12 * ref.S[ok & ~big])


@pytest.mark.parametrize("which", sorted(TABLES))
@pytest.mark.parametrize("launch", [(256, 1280), (128, 16), (64, 4096)])
def test_eam_forces_match_oracle(tb, orc, which, launch):
    """Three wires (1035, 621, 1770 atoms: several tiles and a ragged tail
    each), jittered and moved far from the origin; both precisions on the
    same lists, in the staged, global-fallback and small-tile launch shapes."""
    T = TABLES[which]()
    tab = orc.EamTables(**T)
    b = _batch(0.05, 11)
    b.x = b.x + np.array([1000.0, -350.0, 42.0])
    eng = tb.Engine(b, precision="mixed")
    eng.set_launch(*launch)
    eng.set_eam(**T)
    F32, F64 = eng.forces(f32=True, f64=True)
    F32, F64 = F32.double().cpu().numpy(), F64.cpu().numpy()
    n_amb = 0
    for w in range(b.n_wires):
        s = b.wire_slice(w)
        ref = orc.eam(b.x[s], tab, brute_max=3000)
        amb = ambiguous_atoms(orc, b.x[s], T["r_cut"], 5e-6)
        n_amb += amb.size
        ok = np.ones(b.n[w], bool)
        ok[amb] = False
        d, fm, norm = force_errors(F32[s], ref.F)
        assert np.max(d[ok] / ref.S[ok]) <= 1e-5
        assert norm <= 1e-5
        _check_fp64(F64[s], ref, ambiguous_atoms(orc, b.x[s], T["r_cut"], 1e-10))
    assert n_amb <= 0.05 * b.n_atoms
    eng.close()


@pytest.mark.parametrize("which", sorted(TABLES))
def test_eam_energies_and_virials_match_oracle(tb, orc, which):
    T = TABLES[which]()
    tab = orc.EamTables(**T)
    b = _batch(0.05, 12)
    refs = [orc.eam(b.x[b.wire_slice(w)], tab, brute_max=3000) for w in range(b.n_wires)]
    for prec, tol in (("fp64", 1e-12), ("mixed", 2e-6)):
        eng = tb.Engine(b, precision=prec)
        eng.set_eam(**T)
        e, wv = eng.atom_energies()
        e, wv = e.cpu().numpy(), wv.cpu().numpy()
        for w, ref in enumerate(refs):
            s = b.wire_slice(w)
            amb = ambiguous_atoms(orc, b.x[s], T["r_cut"], 5e-6)
            ok = np.ones(b.n[w], bool)
            ok[amb] = False
            e_ref = ref.eB + ref.eR
            assert np.all(np.abs(e[s][ok] - e_ref[ok]) <= tol * np.abs(e_ref[ok]))
            assert np.all(np.abs(wv[s][ok] - ref.w[ok]) <= tol * 10 * (1 + np.abs(ref.w[ok])))
        eng.close()


def test_embedding_past_the_table_end(tb, orc):
    """A compressed cluster whose densities run past the F table's last
    sample: F continues as its end tangent on both sides of the boundary."""
    T = synthetic(rho_max=20.0)
    tab = orc.EamTables(**T)
    b = workload("tiny_batch")
    eng = tb.Engine(b, precision="fp64")
    eng.set_eam(**T)
    _, F64 = eng.forces(f32=False, f64=True)
    F64 = F64.cpu().numpy()
    s = b.wire_slice(0)
    ref = orc.eam(b.x[s], tab, brute_max=3000)
    assert np.mean(ref.rho > 20.0) > 0.3  # bulk atoms lie past the table
    _check_fp64(F64[s], ref, ambiguous_atoms(orc, b.x[s], T["r_cut"], 1e-10))
    eng.close()


def test_switching_back_to_tbsma_is_exact(tb):
    """set_eam(None) restores Eq. 1-3: the forces equal those of a context
    that never had tables, bit for bit, in both precisions."""
    b = _batch(0.05, 13)
    a = tb.Engine(b, precision="mixed")
    ref32, ref64 = (t.cpu().numpy() for t in a.forces(f32=True, f64=True))
    a.close()
    e = tb.Engine(b, precision="mixed")
    e.set_eam(**synthetic())
    g32, _ = e.forces(f32=True, f64=False)
    assert np.max(np.abs(g32.cpu().numpy() - ref32)) > 1e-3  # the tables acted
    e.set_eam(None)
    g32, g64 = (t.cpu().numpy() for t in e.forces(f32=True, f64=True))
    np.testing.assert_array_equal(g32, ref32)
    np.testing.assert_array_equal(g64, ref64)
    e.close()


def _oracle_vv(orc, tab, x, v, kind, n_steps, dt):
    """Velocity Verlet (B A A B with the halves of the drift as separate
    updates, the integrator's order for gamma = 0) on the oracle's EAM;
    grips (kind > 0) stay fixed at zero strain rate."""
    m = orc.MASS_AU * orc.mvv2e()
    mob = kind == 0
    F = orc.eam(x, tab, brute_max=3000).F
    for _ in range(n_steps):
        v[mob] += 0.5 * dt * F[mob] / m
        x[mob] += 0.5 * dt * v[mob]
        x[mob] += 0.5 * dt * v[mob]
        F = orc.eam(x, tab, brute_max=3000).F
        v[mob] += 0.5 * dt * F[mob] / m
    return x, v


@pytest.mark.parametrize("prec,xtol,vtol", [("fp64", 1e-9, 1e-11), ("mixed", 2e-5, 2e-6)])
def test_eam_md_matches_oracle_short_horizon(tb, orc, prec, xtol, vtol):
    """100 NVE steps (gamma = 0, no pull) of the tiny batch from thermal
    velocities at 10 and 298 K, with the list rebuilt as atoms move: the
    step loop (graph replay, rebuilds, both passes) on the EAM."""
    T = tbsma_sampled()
    tab = orc.EamTables(**T)
    b = workload("tiny_batch")
    b.strain_rate = np.zeros_like(b.strain_rate)
    b.gamma = np.zeros_like(b.gamma)
    v0 = np.zeros_like(b.x)
    for w in range(b.n_wires):
        s = b.wire_slice(w)
        v0[s] = orc.init_velocities(b.kind[s], int(b.seed[w]), float(b.temperature[w]))
    eng = tb.Engine(b, precision=prec)
    eng.set_eam(**T)
    eng.upload(v_host=np.ascontiguousarray(v0.T).reshape(-1))
    eng.step(100, 2.0)
    x, v = eng.positions(), eng.velocities()
    for w in range(b.n_wires):
        s = b.wire_slice(w)
        xo, vo = _oracle_vv(orc, tab, b.x[s].copy(), v0[s].copy(), b.kind[s], 100, 2.0)
        assert np.max(np.abs(x[s] - xo)) < xtol
        assert np.max(np.abs(v[s] - vo)) < vtol
    assert eng.observables()["n_rebuilds"].sum() > 0  # lists were rebuilt on the way
    eng.close()


@pytest.mark.parametrize("prec,xtol,vtol", [("fp64", 1e-9, 1e-11), ("mixed", 2e-5, 2e-6)])
def test_eam_langevin_pull_matches_oracle(tb, orc, prec, xtol, vtol):
    """200 steps of the tiny batch on the EAM with the default protocol on:
    Langevin at 10 and 298 K (Philox normals drawn per atom and step) and
    the grips pulled at 1e9 1/s, against the oracle's BAOAB on its EAM
    (same seeds, same draws).  Positions, velocities, strain, potential
    energy, temperature and stress, as for TB-SMA."""
    T = tbsma_sampled()
    pot = orc.EamPotential(orc.EamTables(**T))
    b = workload("tiny_batch")
    eng = tb.Engine(b, precision=prec)
    eng.set_eam(**T)
    eng.init_velocities()
    v0 = eng.velocities()
    eng.step(200, 2.0)
    x, v = eng.positions(), eng.velocities()
    ob = eng.observables()
    for w in range(b.n_wires):
        s = b.wire_slice(w)
        st = orc.WireState(x=b.x[s].copy(), v=v0[s].copy(), kind=b.kind[s], L0=float(b.L0[w]),
                           strain_rate=float(b.strain_rate[w]),
                           temperature=float(b.temperature[w]), gamma=float(b.gamma[w]),
                           seed=int(b.seed[w]))
        orc.md_steps(st, 200, 2.0, pot=pot, brute_max=3000)
        assert np.max(np.abs(x[s] - st.x)) < xtol
        assert np.max(np.abs(v[s] - st.v)) < vtol
        o = orc.observables(st, pot=pot, brute_max=3000)
        assert o.strain > 0.0
        assert ob["strain"][w] == pytest.approx(o.strain, rel=1e-12)
        assert ob["e_pot"][w] == pytest.approx(o.e_pot, rel=1e-8 if prec == "fp64" else 1e-6)
        assert ob["temp"][w] == pytest.approx(o.temp, rel=1e-6 if prec == "fp64" else 1e-3)
        assert ob["sigma_xx"][w] == pytest.approx(o.sigma_xx, rel=1e-5, abs=1e-7)
        assert ob["n_rebuilds"][w] == st.n_rebuild
    assert ob["temp"][1] > 50.0  # the 298 K wire was thermalised by the draws
    eng.close()


def test_set_eam_rejects_bad_tables(tb):
    T = synthetic()
    eng = tb.Engine(workload("tiny_batch"), precision="mixed")
    bad = [
        dict(T, d_r=0.0),
        dict(T, d_rho=float("nan")),
        dict(T, f=T["f"][:2], phi=T["phi"][:2]),        # 2 samples
        dict(T, f=T["f"][:100], phi=T["phi"][:100]),    # r grid ends before r_cut
        dict(T, phi=np.where(np.arange(T["phi"].size) == 7, np.inf, T["phi"])),
    ]
    before = eng.forces(f32=True, f64=False)[0].cpu().numpy()
    for t in bad:
        with pytest.raises(tb.TbsmaError):
            eng.set_eam(**t)
    # a rejected call leaves the potential as it was
    np.testing.assert_array_equal(eng.forces(f32=True, f64=False)[0].cpu().numpy(), before)
    eng.close()

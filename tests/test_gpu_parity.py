"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances:
  FP64 path  per-atom |dF_i| <= 1e-12 |F_i| (atoms with |F_i| >= 1e-6 S_i),
             else <= 1e-12 S_i; S_i = sum_j |f_ij| is the scale of the pair
             forces on atom i.  Rounding of ~50 FP64 pair terms of size <= S_i
             gives ~1e-15 S_i; libm vs CUDA exp/sqrt differ by <= 2 ulp.
  MIXED path per-atom |dF_i| / S_i <= 1e-5 and ||dF|| / ||F|| <= 1e-5 (the
             force-error target); FP32 pair terms carry ~1e-6 relative error
             (r from rsqrt, exponent argument ~4 r, MUFU ex2), so the bound
             has ~3x margin.
Pairs within a rounding band of r_cut may be decided either way by FP32 (or
by a different FP64 rounding order); atoms whose forces depend on such a
pair are compared at the size of the cutoff jump instead (both answers are
valid), and the test checks that there are few of them.
"""

import math

import numpy as np
import pytest

from inputs import Wire, fcc_wire, jitter, pack, workload
from tests._parity import ambiguous_atoms, force_errors

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def tb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1311_3890_b300 as tb

    tb.lib()
    return tb


def _jittered_batch(sigma=0.05, seed=0):
    b = workload("tiny_batch")
    b.x = jitter(b.x, sigma, seed)
    return b


def _oracle_forces(orc, b):
    return [orc.tbsma(b.x[b.wire_slice(w)], brute_max=3000) for w in range(b.n_wires)]


# ------------------------------------------------------------------ Philox
def test_philox_bitwise_equals_oracle(tb, orc):
    rng = np.random.default_rng(5)
    n = 4096
    ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2**32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    key[0] = 0
    ctr[1] = 0xFFFFFFFF
    key[1] = 0xFFFFFFFF
    got = tb.philox4x32_10(torch.from_numpy(ctr.view(np.int32)).cuda(),
                           torch.from_numpy(key.view(np.int32)).cuda())
    torch.cuda.synchronize()
    got = got.cpu().numpy().view(np.uint32)
    ref = orc.philox4x32_10(ctr, key)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("step", [0, 17, (1 << 33) + 5])
def test_normals_match_oracle(tb, orc, step):
    n = 200_000
    atoms = np.arange(n, dtype=np.uint32)
    ref = orc.normals(1234567, atoms, step, 0)
    at = torch.from_numpy(atoms.view(np.int32)).cuda()
    g64 = tb.normals(1234567, at, step, 0, "fp64").cpu().numpy()
    g32 = tb.normals(1234567, at, step, 0, "mixed").cpu().numpy()
    # FP64 Box-Muller: libm vs CUDA log/sqrt/sincos differ by a few ulp
    assert np.max(np.abs(g64 - ref)) < 1e-13
    # FP32 Box-Muller: u1 rounded to FP32 moves the angle by <= 2pi 2^-25
    assert np.max(np.abs(g32 - ref) / (1.0 + np.abs(ref))) < 2e-6


# ------------------------------------------------------------------ forces
def _check_fp64(F, ref, amb):
    d, fm, _ = force_errors(F, ref.F)
    ok = np.ones(F.shape[0], bool)
    ok[amb] = False
    big = ok & (fm >= 1e-6 * ref.S)
    assert np.all(d[big] <= 1e-12 * fm[big])
    assert np.all(d[ok & ~big] <= 1e-12 * ref.S[ok & ~big])
    return d


@pytest.mark.parametrize("block,window", [(64, 0), (128, 2048), (256, 512)])
def test_forces_fp64_match_oracle(tb, orc, block, window):
    b = _jittered_batch()
    eng = tb.Engine(b, precision="fp64")
    eng.set_launch(block, window)
    _, F64 = eng.forces(f32=False, f64=True)
    F64 = F64.cpu().numpy()
    for w, ref in enumerate(_oracle_forces(orc, b)):
        s = b.wire_slice(w)
        _check_fp64(F64[s], ref, ambiguous_atoms(orc, b.x[s], orc.AU.r_cut, 1e-10))
    eng.close()


@pytest.mark.parametrize("sigma,seed", [(0.02, 1), (0.05, 2), (0.12, 3)])
def test_forces_mixed_match_oracle(tb, orc, sigma, seed):
    b = _jittered_batch(sigma, seed)
    # far from the origin: fixed point is relative to each wire's centre
    b.x = b.x + np.array([1000.0, -350.0, 42.0])
    eng = tb.Engine(b, precision="mixed")
    # staged window, global fallback (window too small), tiles of 64
    eng.set_launch(*[(256, 2048), (128, 16), (64, 4096)][seed - 1])
    F32, F64 = eng.forces(f32=True, f64=True)
    F32, F64 = F32.double().cpu().numpy(), F64.cpu().numpy()
    n_amb = 0
    for w, ref in enumerate(_oracle_forces(orc, b)):
        s = b.wire_slice(w)
        amb = ambiguous_atoms(orc, b.x[s], orc.AU.r_cut, 5e-6)
        n_amb += amb.size
        ok = np.ones(b.n[w], bool)
        ok[amb] = False
        d, fm, norm = force_errors(F32[s], ref.F)
        assert np.max(d[ok] / ref.S[ok]) <= 1e-5
        assert norm <= 1e-5
        # an ambiguous pair moves a force by at most the cutoff jump (< 1e-3 eV/A)
        assert np.all(d[amb] < 1e-3)
        _check_fp64(F64[s], ref, ambiguous_atoms(orc, b.x[s], orc.AU.r_cut, 1e-10))
    assert n_amb <= 0.05 * b.n_atoms
    eng.close()


def test_energies_and_virials_match_oracle(tb, orc):
    b = _jittered_batch(0.05, 7)
    refs = _oracle_forces(orc, b)
    for prec, tol in (("fp64", 1e-12), ("mixed", 2e-6)):
        eng = tb.Engine(b, precision=prec)
        e, wv = eng.atom_energies()
        e, wv = e.cpu().numpy(), wv.cpu().numpy()
        for w, ref in enumerate(refs):
            s = b.wire_slice(w)
            amb = ambiguous_atoms(orc, b.x[s], orc.AU.r_cut, 5e-6)
            ok = np.ones(b.n[w], bool)
            ok[amb] = False
            e_ref = ref.eB + ref.eR
            assert np.all(np.abs(e[s][ok] - e_ref[ok]) <= tol * np.abs(e_ref[ok]))
            assert np.all(np.abs(wv[s][ok] - ref.w[ok]) <= tol * 10 * (1 + np.abs(ref.w[ok])))
        eng.close()


def test_neighbor_lists_bracket_oracle_pairs(tb, orc):
    b = _jittered_batch(0.08, 9)
    eng = tb.Engine(b, precision="mixed")
    n, nb = eng.neighbors()
    n, nb = n.cpu().numpy(), nb.cpu().numpy()
    r_list = orc.AU.r_cut + orc.R_SKIN + 1e-3
    for w in range(b.n_wires):
        s = b.wire_slice(w)
        o = int(b.offset[w])
        s_in, n_in = orc.pairs(b.x[s], r_list - 1e-4)
        s_out, n_out = orc.pairs(b.x[s], r_list + 1e-4)
        for i in range(int(b.n[w])):
            got = set((nb[o + i, :n[o + i]] - o).tolist())
            assert set(n_in[s_in[i]:s_in[i + 1]].tolist()) <= got
            assert got <= set(n_out[s_out[i]:s_out[i + 1]].tolist())
    eng.close()


def test_disordered_atom_order_takes_the_cell_build(tb, orc):
    """One wire's atoms in random order: its envelopes along the atom order
    are far apart, so the library builds its lists through the cell grid
    instead of the slab scan.  Both builds accept a pair at d <= r_list, the
    cell build on exact fixed-point differences, the slab scan on FP32
    coordinates (within a few 1e-6 A here), so that wire's lists hold the
    same atoms as those of the same wire in [100] order (a slab build) but
    for pairs within 1e-4 A of r_list; its lists bracket the oracle's pairs,
    and its forces match the oracle's."""
    b = _jittered_batch(0.05, 29)
    w = 1
    s = b.wire_slice(w)
    p = np.random.default_rng(4).permutation(int(b.n[w]))
    b2 = _jittered_batch(0.05, 29)
    b2.x[s] = b.x[s][p]
    b2.kind[s] = b.kind[s][p]
    o = int(b.offset[w])
    rows = []
    for bb in (b, b2):
        eng = tb.Engine(bb, precision="mixed")
        n, nb = eng.neighbors()
        F32, _ = eng.forces(f32=True, f64=False)
        rows.append((n.cpu().numpy(), nb.cpu().numpy(), F32.double().cpu().numpy()))
        eng.close()
    (n1, nb1, _), (n2, nb2, F2) = rows
    r_list = orc.AU.r_cut + orc.R_SKIN + 1e-3
    xs = b.x[s]
    for k in range(int(b.n[w])):
        got = {int(p[j - o]) for j in nb2[o + k, :n2[o + k]]}
        ref = set((nb1[o + p[k], :n1[o + p[k]]] - o).tolist())
        for j in got ^ ref:
            assert abs(np.linalg.norm(xs[j] - xs[p[k]]) - r_list) < 1e-4
    s_in, n_in = orc.pairs(b2.x[s], r_list - 1e-4)
    for k in range(int(b.n[w])):
        assert set(n_in[s_in[k]:s_in[k + 1]].tolist()) <= set((nb2[o + k, :n2[o + k]] - o).tolist())
    ref = orc.tbsma(b2.x[s], brute_max=3000)
    amb = ambiguous_atoms(orc, b2.x[s], orc.AU.r_cut, 5e-6)
    ok = np.ones(int(b.n[w]), bool)
    ok[amb] = False
    d, fm, norm = force_errors(F2[s], ref.F)
    assert np.max(d[ok] / ref.S[ok]) <= 1e-5
    assert norm <= 1e-5


@pytest.mark.parametrize("long_first", [True, False])
def test_wire_beyond_the_slab_coordinate_range_takes_the_cell_build(tb, orc, long_first):
    """A D2 x 300 nm wire (55k atoms) moved 600 A along its axis after init
    reaches 2100 A from its fixed-point origin, beyond the 2048 A within
    which the slab scan's FP32 coordinates stay inside the list radius's
    guard, so its lists come from the cell grid (whose +L/2 margins hold the
    moved wire); the short wire beside it takes the slab scan.  Both wires'
    lists bracket the oracle's pairs and their forces match the oracle's,
    with the cell-built wire first or second in the batch (the cell build
    walks its own compacted list of wires)."""
    geoms = (fcc_wire(2.0, 300.0), fcc_wire(2.0, 6.0))
    if not long_first:
        geoms = geoms[::-1]
    wires = [Wire(x=jitter(g.x, 0.05, 31 + k), kind=g.kind, diameter_nm=2.0, length_nm=g.length_nm,
                  L0=g.L0, temperature=10.0, strain_rate=0.0, gamma=1e-3, seed=k)
             for k, g in enumerate(geoms)]
    b = pack(wires)
    eng = tb.Engine(b, precision="mixed")
    s0 = b.wire_slice(0 if long_first else 1)
    origin = 0.5 * (b.x[s0, 0].min() + b.x[s0, 0].max())  # the centre of the initial box
    b.x[s0, 0] += 600.0
    assert np.max(np.abs(b.x[s0, 0] - origin)) > 2048.0
    eng.upload(np.ascontiguousarray(b.x.T).reshape(-1), None)
    eng.build_neighbors(True)
    n, nb = eng.neighbors()
    n, nb = n.cpu().numpy(), nb.cpu().numpy()
    F32, _ = eng.forces(f32=True, f64=False)
    F32 = F32.double().cpu().numpy()
    assert np.all(eng.wire_status() == 0)
    eng.close()
    r_list = orc.AU.r_cut + orc.R_SKIN + 1e-3
    for w in range(2):
        s = b.wire_slice(w)
        o = int(b.offset[w])
        s_in, n_in = orc.pairs(b.x[s], r_list - 1e-4, "cells")
        for k in range(int(b.n[w])):
            assert set(n_in[s_in[k]:s_in[k + 1]].tolist()) <= set((nb[o + k, :n[o + k]] - o).tolist())
        ref = orc.tbsma(b.x[s], brute_max=0)
        amb = ambiguous_atoms(orc, b.x[s], orc.AU.r_cut, 5e-6)
        ok = np.ones(int(b.n[w]), bool)
        ok[amb] = False
        d, fm, norm = force_errors(F32[s], ref.F)
        assert np.max(d[ok] / ref.S[ok]) <= 1e-5
        assert norm <= 1e-5


# --------------------------------------------------------- initial state
def test_init_velocities_match_oracle(tb, orc):
    b = workload("tiny_batch")
    eng = tb.Engine(b, precision="fp64")
    eng.init_velocities()
    v = eng.velocities()
    for w in range(b.n_wires):
        s = b.wire_slice(w)
        ref = orc.init_velocities(b.kind[s], int(b.seed[w]), float(b.temperature[w]))
        assert np.max(np.abs(v[s] - ref)) < 1e-14
    ob = eng.observables()
    assert np.allclose(ob["temp"], b.temperature, rtol=1e-12)
    eng.close()


# ----------------------------------------------------------- trajectories
def _oracle_run(orc, b, w, v0, n_steps, dt=2.0):
    s = b.wire_slice(w)
    st = orc.WireState(x=b.x[s].copy(), v=v0[s].copy(), kind=b.kind[s], L0=float(b.L0[w]),
                       strain_rate=float(b.strain_rate[w]), temperature=float(b.temperature[w]),
                       gamma=float(b.gamma[w]), seed=int(b.seed[w]))
    orc.md_steps(st, n_steps, dt, brute_max=3000)
    return st


@pytest.mark.parametrize("prec,xtol,vtol", [("fp64", 1e-9, 1e-11), ("mixed", 2e-5, 2e-6)])
def test_md_matches_oracle_short_horizon(tb, orc, prec, xtol, vtol):
    """200 steps (0.4 ps) of the tiny batch at 10 and 298 K with the pull on.
    FP64: the paths differ by rounding order only.  MIXED: FP32 forces
    (~1e-6 relative) and FP32 Box-Muller normals (~1e-6) perturb a chaotic
    trajectory; over 0.4 ps the divergence stays below the bounds."""
    b = workload("tiny_batch")
    eng = tb.Engine(b, precision=prec)
    eng.init_velocities()
    v0 = eng.velocities()
    eng.step(200, 2.0)
    x, v = eng.positions(), eng.velocities()
    ob = eng.observables()
    for w in range(b.n_wires):
        s = b.wire_slice(w)
        st = _oracle_run(orc, b, w, v0, 200)
        assert np.max(np.abs(x[s] - st.x)) < xtol
        assert np.max(np.abs(v[s] - st.v)) < vtol
        o = orc.observables(st, brute_max=3000)
        assert ob["strain"][w] == pytest.approx(o.strain, rel=1e-12)
        assert ob["e_pot"][w] == pytest.approx(o.e_pot, rel=1e-8 if prec == "fp64" else 1e-6)
        assert ob["temp"][w] == pytest.approx(o.temp, rel=1e-6 if prec == "fp64" else 1e-3)
        assert ob["sigma_xx"][w] == pytest.approx(o.sigma_xx, rel=1e-5, abs=1e-7)
        assert ob["n_rebuilds"][w] == st.n_rebuild
    assert np.all(ob["step"] == 200)
    eng.close()


def _wire_of(b, w):
    s = b.wire_slice(w)
    return Wire(x=b.x[s].copy(), kind=b.kind[s].copy(), diameter_nm=0.0, length_nm=0.0,
                L0=float(b.L0[w]), temperature=float(b.temperature[w]),
                strain_rate=float(b.strain_rate[w]), gamma=float(b.gamma[w]), seed=int(b.seed[w]))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_equals_single_wires_bitwise(tb, prec):
    b = workload("tiny_batch")
    eng = tb.Engine(b, precision=prec)
    eng.init_velocities()
    eng.step(120, 2.0)
    x, v = eng.positions(), eng.velocities()
    eng.close()
    for w in range(b.n_wires):
        s = b.wire_slice(w)
        e1 = tb.Engine(pack([_wire_of(b, w)]), precision=prec)
        e1.init_velocities()
        e1.step(120, 2.0)
        assert np.array_equal(e1.positions(), x[s])
        assert np.array_equal(e1.velocities(), v[s])
        e1.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_rerun_and_chunking_are_deterministic(tb, prec):
    b = workload("tiny_batch")
    runs = []
    for split in ((120,), (50, 70), (120,)):
        eng = tb.Engine(b, precision=prec)
        eng.init_velocities()
        for n in split:
            eng.step(n, 2.0)
        runs.append((eng.positions(), eng.velocities()))
        eng.close()
    for x, v in runs[1:]:
        assert np.array_equal(x, runs[0][0]) and np.array_equal(v, runs[0][1])


def test_observables_static_match_oracle(tb, orc):
    b = _jittered_batch(0.03, 11)
    eng = tb.Engine(b, precision="fp64")
    ob = eng.observables()
    for w in range(b.n_wires):
        s = b.wire_slice(w)
        st = orc.WireState(x=b.x[s], v=np.zeros_like(b.x[s]), kind=b.kind[s], L0=float(b.L0[w]))
        o = orc.observables(st, brute_max=3000)
        assert ob["e_pot"][w] == pytest.approx(o.e_pot, rel=1e-12)
        assert ob["virial_xx"][w] == pytest.approx(o.virial_xx, rel=1e-10, abs=1e-10)
        assert ob["sigma_xx"][w] == pytest.approx(o.sigma_xx, rel=1e-10, abs=1e-12)
        assert ob["strain"][w] == 0.0 and ob["status"][w] == 0
    eng.close()


def test_force_check_api(tb):
    b = _jittered_batch(0.05, 13)
    eng = tb.Engine(b, precision="mixed")
    fc = eng.force_check()
    F32, F64 = eng.forces(f32=True, f64=True)
    F32, F64 = F32.double().cpu().numpy(), F64.cpu().numpy()
    for w in range(b.n_wires):
        s = b.wire_slice(w)
        d, fm, norm = force_errors(F32[s], F64[s])
        assert fc["norm_err"][w] == pytest.approx(norm, rel=1e-9)
        assert fc["max_abs_err"][w] == pytest.approx(d.max(), rel=1e-9)
        assert fc["max_err_scaled"][w] <= 1e-5
    eng.close()


def test_upload_download_roundtrip(tb):
    b = workload("tiny_batch")
    eng = tb.Engine(b, precision="mixed")
    eng.init_velocities()
    xh = np.zeros(3 * b.n_atoms)
    vh = np.zeros(3 * b.n_atoms)
    eng.download(xh, vh)
    assert np.array_equal(xh.reshape(3, -1).T, b.x)
    eng.step(10)
    x1 = eng.positions()
    eng.upload(xh, vh)  # back to the start; lists and forces are refreshed
    eng.step(10)
    assert np.all(np.isfinite(eng.positions()))
    eng.download(xh, None)
    assert np.array_equal(xh.reshape(3, -1).T, eng.positions())
    # the thermostat counter kept running, so the second 10 steps draw new noise
    assert not np.array_equal(x1, eng.positions())
    eng.close()


# ------------------------------------------------------------- edge cases
def test_isolated_atom_and_dimer_wires(tb, orc):
    from inputs import dimer

    P = orc.AU
    r = 2.5
    w1 = Wire(x=np.array([[0.0, 0.0, 0.0]]), kind=np.zeros(1, np.uint8), diameter_nm=0,
              length_nm=0, L0=1.0)
    w2 = Wire(x=dimer(r) + 30.0, kind=np.zeros(2, np.uint8), diameter_nm=0, length_nm=0, L0=1.0)
    b = pack([w1, w2])
    sE = r / P.r0 - 1
    closed = 2 * P.A * math.exp(-P.p * sE) - 2 * P.xi * math.exp(-P.q * sE)
    for prec, tol in (("fp64", 1e-13), ("mixed", 3e-6)):
        eng = tb.Engine(b, precision=prec)
        ob = eng.observables()
        assert ob["e_pot"][0] == 0.0
        assert ob["e_pot"][1] == pytest.approx(closed, rel=tol)
        F32, F64 = eng.forces()
        F = (F32.double() if prec == "mixed" else F64).cpu().numpy()
        assert np.all(F[0] == 0)
        assert F[1, 0] == pytest.approx(orc.tbsma(dimer(r)).F[0, 0], rel=tol)
        eng.step(5)
        eng.close()


def test_invalid_arguments_rejected(tb):
    b = workload("tiny_batch")
    b.n = b.n.copy()
    b.n[1] = 0
    with pytest.raises(tb.TbsmaError) as e:
        tb.Engine(b)
    assert e.value.status == 1
    eng = tb.Engine(workload("tiny_batch"))
    with pytest.raises(tb.TbsmaError):
        eng.step(5, dt=-1.0)
    with pytest.raises(tb.TbsmaError):
        eng.set_launch(3, 128)
    eng.close()


def test_nonfinite_wire_is_flagged_and_others_continue(tb):
    b = workload("tiny_batch")
    ref = tb.Engine(b, precision="mixed")
    ref.init_velocities()
    ref.step(20)
    x_ref = ref.positions()
    ref.close()
    eng = tb.Engine(b, precision="mixed")
    eng.init_velocities()
    # poison one coordinate of wire 1 through the host upload path
    xh = np.zeros(3 * b.n_atoms)
    eng.download(xh, None)
    xh[int(b.offset[1]) + 5] = np.nan
    eng.upload(xh, None)
    st = eng.step(20, check=False)
    assert st == 6  # TBSMA_EWIRE
    status = eng.wire_status()
    assert status[1] & 1 and status[0] == 0 and status[2] == 0
    x = eng.positions()
    for w in (0, 2):
        s = b.wire_slice(w)
        assert np.array_equal(x[s], x_ref[s])
    eng.close()


def test_neighbor_overflow_is_reported(tb):
    # a compressed lattice (a = 3.2 A) has > 64 neighbours inside 6.09 A
    w = fcc_wire(2.0, 3.0, a=3.2)
    with pytest.raises(tb.TbsmaError) as e:
        eng = tb.Engine(pack([w]))
        eng.build_neighbors(force_all=True)
    assert e.value.status == 4  # TBSMA_EOVERFLOW


# --------------------------------------------- full size, bench configuration
def test_full_size_batch_sampled_against_oracle(tb, orc):
    """The 256-wire D3 x L40 batch (4.46M atoms) in the bench's launch shape:
    every wire's net force vanishes, and three sampled wires match the oracle
    atom by atom."""
    from bench import LAUNCH

    b = workload("batch256_d3_l40")
    b.x = jitter(b.x, 0.03, 21)
    eng = tb.Engine(b, precision="mixed")
    eng.set_launch(*LAUNCH)
    F32, _ = eng.forces(f32=True, f64=False)
    F32 = F32.double().cpu().numpy()
    for w in range(b.n_wires):
        s = b.wire_slice(w)
        net = np.abs(F32[s].sum(axis=0)).max()
        assert net < 1e-6 * np.abs(F32[s]).sum()
    for w in (0, 137, 255):
        s = b.wire_slice(w)
        ref = orc.tbsma(b.x[s], brute_max=0)
        amb = ambiguous_atoms(orc, b.x[s], orc.AU.r_cut, 5e-6)
        ok = np.ones(b.n[w], bool)
        ok[amb] = False
        d, fm, norm = force_errors(F32[s], ref.F)
        assert np.max(d[ok] / ref.S[ok]) <= 1e-5
        assert norm <= 1e-5
    eng.close()


def test_full_size_sweep_sampled_against_oracle(tb, orc):
    """The bench workload, the 2048-wire sweep (55.8M atoms, D 2-4 nm, L 5-120
    nm), jittered, in the bench's launch shape and list skin: every wire's
    net force vanishes, and the smallest and the largest wire of each
    diameter match the oracle atom by atom."""
    from bench import LAUNCH, R_SKIN
    from inputs.configs import WORKLOADS

    specs = WORKLOADS["sweep2048"]()
    b = workload("sweep2048")
    b.x = jitter(b.x, 0.05, 23)
    eng = tb.Engine(b, precision="mixed", params=tb.au_params(r_skin=R_SKIN))
    eng.set_launch(*LAUNCH)
    F32, _ = eng.forces(f32=True, f64=False)
    F32 = F32.double().cpu().numpy()
    eng.close()
    for w in range(b.n_wires):
        s = b.wire_slice(w)
        net = np.abs(F32[s].sum(axis=0)).max()
        assert net < 1e-6 * np.abs(F32[s]).sum()
    picks = []
    for d in (2.0, 3.0, 4.0):
        ws = [w for w, sp in enumerate(specs) if sp.diameter_nm == d]
        picks += [min(ws, key=lambda w: b.n[w]), max(ws, key=lambda w: b.n[w])]
    for w in picks:
        s = b.wire_slice(w)
        ref = orc.tbsma(b.x[s], brute_max=0)
        amb = ambiguous_atoms(orc, b.x[s], orc.AU.r_cut, 5e-6)
        ok = np.ones(b.n[w], bool)
        ok[amb] = False
        d, fm, norm = force_errors(F32[s], ref.F)
        assert np.max(d[ok] / ref.S[ok]) <= 1e-5
        assert norm <= 1e-5


def test_force_error_gate_on_thermalised_wires(tb, orc):
    """The mixed-precision force check (same positions, same list, same
    cutoff decisions) on 8 D3 x L40 wires after 1000 steps at 10 K, where
    near-equilibrium forces are smallest relative to their pair terms, and
    one of those wires against the oracle."""
    from inputs.configs import WORKLOADS, build

    b = build(WORKLOADS["batch256_d3_l40"]()[:8])
    eng = tb.Engine(b, precision="mixed")
    eng.init_velocities()
    eng.step(1000, 2.0)
    fc = eng.force_check()
    assert fc["max_err_scaled"].max() <= 1e-5
    assert fc["norm_err"].max() <= 1e-5
    x = eng.positions()
    F32, _ = eng.forces(f32=True, f64=False)
    F32 = F32.double().cpu().numpy()
    s = b.wire_slice(3)
    ref = orc.tbsma(x[s], brute_max=0)
    amb = ambiguous_atoms(orc, x[s], orc.AU.r_cut, 5e-6)
    ok = np.ones(int(b.n[3]), bool)
    ok[amb] = False
    d, fm, _ = force_errors(F32[s], ref.F)
    assert np.max(d[ok] / ref.S[ok]) <= 1e-5
    assert np.linalg.norm(d[ok]) <= 1e-5 * np.linalg.norm(fm[ok])
    eng.close()


def test_launch_shape_never_changes_forces_and_autotuner_picks_one(tb, tmp_path):
    from paper_1311_3890_b300.autotune import CANDIDATES, tune

    b = _jittered_batch(0.05, 17)
    eng = tb.Engine(b, precision="mixed")
    ref = None
    for blk, win in CANDIDATES + [(64, 16)]:
        eng.set_launch(blk, win)
        F32, F64 = eng.forces(f32=True, f64=True)
        cur = (F32.cpu().numpy(), F64.cpu().numpy())
        if ref is None:
            ref = cur
        assert np.array_equal(cur[0], ref[0]) and np.array_equal(cur[1], ref[1])
    cache = tmp_path / "tune.json"
    best, entry = tune(eng, cache_path=str(cache), reps=2)
    assert tuple(best) in CANDIDATES and cache.exists()
    again, _ = tune(eng, cache_path=str(cache))
    assert tuple(again) == tuple(best)
    eng.close()

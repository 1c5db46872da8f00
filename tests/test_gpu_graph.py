"""Captured step graphs against directly enqueued steps: a call of n steps
replays a captured graph of min(n, 50) steps as often as it fits and
enqueues the remainder directly; both must give the same trajectory bit for
bit, and the library's count of rebuild-chain launches (the bench's launch
accounting) must be one per step and per position refresh.
"""

import numpy as np
import pytest

from inputs import workload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def tb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1311_3890_b300 as tb

    tb.lib()
    return tb


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_graph_and_direct_steps_agree_bitwise(tb, prec):
    """300 steps of the tiny batch (10 K and 298 K wires, pulled) as calls
    of 50 and 25 steps, each a captured graph, and as calls of 75 steps, a
    50-step graph replay followed by 25 directly enqueued steps: the kicks
    are split at the same steps (every call and every graph replay ends with
    its closing half kick), so positions, velocities and rebuild counts
    must agree bit for bit."""
    b = workload("tiny_batch")
    out = []
    for split in ([50, 25] * 4, [75] * 4):
        eng = tb.Engine(b, precision=prec)
        eng.set_step_mode("graph")
        eng.init_velocities()
        for n in split:
            eng.step(n, 2.0)
        ob = eng.observables()
        out.append((eng.positions(), eng.velocities(), ob["n_rebuilds"].copy(),
                    eng.rebuild_chains()))
        eng.close()
    (xa, va, ra, ca), (xb, vb, rb, cb) = out
    np.testing.assert_array_equal(xa, xb)
    np.testing.assert_array_equal(va, vb)
    np.testing.assert_array_equal(ra, rb)
    assert ra.sum() > 3  # the wires did rebuild
    # one chain per step, plus the two builds of init and the report's refresh
    assert ca == cb == 300 + 3


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_profiled_steps_equal_graph_steps(tb, prec):
    """tbsma_step_profile enqueues the same kernels in the same order as the
    graph replays, only with an event after each phase: 120 profiled steps
    (sequences of 50, 50 and 20) equal 120 steps of one step call bit for
    bit, with the same list builds; the phase times are positive where the
    phase does work, and the list-build accounting counts the init's two
    full builds of every wire."""
    b = workload("tiny_batch")
    out = []
    for profiled in (False, True):
        eng = tb.Engine(b, precision=prec)
        eng.set_step_mode("graph")
        rs = eng.rebuild_stats()
        assert rs == {"chains": 2, "wires": 2 * b.n_wires, "atoms": 2 * b.n_atoms}
        eng.init_velocities()
        ph = eng.step_profile(120, 2.0) if profiled else eng.step(120, 2.0)
        out.append((eng.positions(), eng.velocities(), eng.rebuild_stats(), ph))
        eng.close()
    (xa, va, ra, _), (xb, vb, rb, ph) = out
    np.testing.assert_array_equal(xa, xb)
    np.testing.assert_array_equal(va, vb)
    assert ra == rb and ra["chains"] == 2 + 120 and ra["wires"] > 2 * b.n_wires
    assert set(ph) == {"integrate", "plan", "rebuild", "density", "force", "kick"}
    assert all(v > 0.0 for v in ph.values())


@pytest.mark.parametrize("lanes", [1, 2, 4])
def test_persistent_step_kernel_equals_graph_replays(tb, lanes):
    """The persistent step kernel (one cooperative launch per call, grid
    barriers between the phases) runs the graph path's code per atom and
    per tile: 300 steps of the tiny batch (10 K and 298 K wires, pulled,
    with list rebuilds) in calls of 50 and 25 steps give bitwise the
    positions, velocities, rebuild counts and list-build accounting of
    graph replays, and the observables after them agree."""
    b = workload("tiny_batch")
    out = []
    for mode in ("graph", "persistent"):
        eng = tb.Engine(b, precision="mixed")
        if mode == "persistent":
            eng.set_pair_lanes(lanes)
        blocks = eng.set_step_mode(mode)
        if mode == "persistent":  # one block per pair-pass tile of 256 / lanes atoms
            assert blocks == lanes * int(np.sum((b.n + 255) // 256))
        eng.init_velocities()
        for n in [50, 25] * 4:
            eng.step(n, 2.0)
        ob = eng.observables()
        out.append((eng.positions(), eng.velocities(), ob, eng.rebuild_stats()))
        eng.close()
    (xa, va, oa, ra), (xb, vb, ob, rb) = out
    np.testing.assert_array_equal(xa, xb)
    np.testing.assert_array_equal(va, vb)
    np.testing.assert_array_equal(oa["n_rebuilds"], ob["n_rebuilds"])
    assert oa["n_rebuilds"].sum() > 3  # the wires did rebuild
    assert ra == rb
    for k in ("e_pot", "e_kin", "sigma_xx", "strain"):
        np.testing.assert_array_equal(oa[k], ob[k])


def test_persistent_step_kernel_with_a_cell_built_wire_equals_graph_replays(tb):
    """A batch whose second wire has its atoms in random order (its lists
    come from the cell build, the others' from the slab scan; both builds
    use the kernel's shared memory, after which each block reloads its tile
    cache): 200 steps at 298 K in the persistent kernel equal graph replays
    bitwise, with rebuilds on the way."""
    b = workload("tiny_batch")
    b.temperature[:] = 298.0
    s = b.wire_slice(1)
    p = np.random.default_rng(8).permutation(int(b.n[1]))
    b.x[s] = b.x[s][p]
    b.kind[s] = b.kind[s][p]
    out = []
    for mode in ("graph", "persistent"):
        eng = tb.Engine(b, precision="mixed")
        assert (eng.set_step_mode(mode) > 0) == (mode == "persistent")
        eng.init_velocities()
        for n in (50, 50, 100):
            eng.step(n, 2.0)
        out.append((eng.positions(), eng.velocities(), eng.observables()["n_rebuilds"]))
        eng.close()
    (xa, va, na), (xb, vb, nb) = out
    np.testing.assert_array_equal(xa, xb)
    np.testing.assert_array_equal(va, vb)
    np.testing.assert_array_equal(na, nb)
    assert na[1] > 0  # the shuffled wire was rebuilt


def test_persistent_barrier_gives_up_and_context_recovers(tb, tmp_path):
    """Failure detection of the persistent step kernel without a fault: with
    the wait limit at 1 every block that is not the last to reach a grid
    barrier gives up at once, every block leaves, and the step call returns
    TBSMA_ETIMEOUT.  With the limit restored, the same context resumes from
    a checkpoint and continues bit for bit as a context that never timed
    out."""
    b = workload("tiny_batch")
    eng = tb.Engine(b, precision="mixed")
    assert eng.set_step_mode("persistent") > 1
    eng.init_velocities()
    eng.step(100, 2.0)
    ck = str(tmp_path / "ck")
    eng.save(ck)
    eng.set_wait_limit(1)
    with pytest.raises(tb.TbsmaError) as e:
        eng.step(20, 2.0)
    assert e.value.status == 5  # TBSMA_ETIMEOUT
    eng.set_wait_limit(1 << 20)
    eng.load(ck)
    eng.step(100, 2.0)
    x1, v1 = eng.positions(), eng.velocities()
    eng.close()
    ref = tb.Engine(b, precision="mixed")
    ref.set_step_mode("persistent")
    ref.load(ck)
    ref.step(100, 2.0)
    np.testing.assert_array_equal(ref.positions(), x1)
    np.testing.assert_array_equal(ref.velocities(), v1)
    ref.close()


def test_persistent_mode_is_refused_where_it_cannot_run(tb):
    """The paper's protocol mode and launch shapes other than 256-atom tiles
    run graph replays; asking them for the persistent step kernel is an
    EINVAL at the step call."""
    b = workload("tiny_batch")
    for prec in ("mixed", "fp64"):
        eng = tb.Engine(b, precision=prec)
        eng.set_protocol()
        assert eng.set_step_mode("persistent") == 0
        with pytest.raises(tb.TbsmaError) as e:
            eng.step(5, 2.0)
        assert e.value.status == 1
        eng.close()
    eng = tb.Engine(b, precision="mixed")
    eng.set_launch(64, 1280)
    assert eng.set_step_mode("auto") == 0
    eng.step(5, 2.0)  # graph replays
    eng.close()


def test_fp64_persistent_step_kernel_equals_graph_replays(tb):
    """FP64 contexts run the persistent step kernel too (16 lanes per slot in
    the FP64 passes, the cell build on rebuilds): 300 steps of the tiny batch
    (10 K and 298 K, pulled, with rebuilds) in calls of 50 and 25 steps give
    bitwise the positions, velocities and rebuild counts of graph replays."""
    b = workload("tiny_batch")
    out = []
    for mode in ("graph", "persistent"):
        eng = tb.Engine(b, precision="fp64")
        blocks = eng.set_step_mode(mode)
        assert (blocks > 0) == (mode == "persistent")
        eng.init_velocities()
        for n in [50, 25] * 4:
            eng.step(n, 2.0)
        ob = eng.observables()
        out.append((eng.positions(), eng.velocities(), ob, eng.rebuild_stats()))
        eng.close()
    (xa, va, oa, ra), (xb, vb, ob, rb) = out
    np.testing.assert_array_equal(xa, xb)
    np.testing.assert_array_equal(va, vb)
    np.testing.assert_array_equal(oa["n_rebuilds"], ob["n_rebuilds"])
    assert oa["n_rebuilds"].sum() > 3
    assert ra == rb
    for k in ("e_pot", "e_kin", "sigma_xx", "strain"):
        np.testing.assert_array_equal(oa[k], ob[k])


def test_fp64_persistent_step_kernel_on_more_atoms_than_threads(tb):
    """Six D3 x L40 wires (~105k atoms, 10 and 298 K, pulled) in FP64: more
    atoms than the persistent grid has threads, so the integrate loops'
    8-atom chunks take a second round and every block owns several slots of
    the FP64 passes; 100 steps with rebuilds give bitwise the graph
    replays' positions, velocities and rebuild counts."""
    from inputs.configs import WireSpec, build

    b = build([WireSpec(3.0, 40.0, 10.0 if s % 2 == 0 else 298.0, 1.0e9, s) for s in range(6)])
    out = []
    for mode in ("graph", "persistent"):
        eng = tb.Engine(b, precision="fp64")
        blocks = eng.set_step_mode(mode)
        if mode == "persistent":
            assert 0 < blocks * 128 < b.n_atoms
        eng.init_velocities()
        for n in (50, 25, 25):
            eng.step(n, 2.0)
        ob = eng.observables()
        out.append((eng.positions(), eng.velocities(), ob, eng.rebuild_stats()))
        eng.close()
    (xa, va, oa, ra), (xb, vb, ob, rb) = out
    np.testing.assert_array_equal(xa, xb)
    np.testing.assert_array_equal(va, vb)
    np.testing.assert_array_equal(oa["n_rebuilds"], ob["n_rebuilds"])
    assert oa["n_rebuilds"].sum() > 0
    assert ra == rb


def test_two_and_four_lanes_per_atom_give_bitwise_the_same_results(tb):
    """The pair passes with two or four threads per atom (each evaluating
    every second or fourth entry of every group of four, the terms added in
    list order through shuffles) give bitwise the forces, energies and
    virials of one thread per atom on a jittered tiny batch, and the same
    trajectory."""
    from inputs import jitter

    b = workload("tiny_batch")
    b.x = jitter(b.x, 0.06, 41)
    out = []
    for lanes in (1, 2, 4):
        eng = tb.Engine(b, precision="mixed")
        eng.set_step_mode("graph")
        eng.set_pair_lanes(lanes)
        F32, _ = eng.forces(f32=True, f64=False)
        e, w = eng.atom_energies()
        eng.init_velocities()
        eng.step(120, 2.0)
        out.append((F32.cpu().numpy(), e.cpu().numpy(), w.cpu().numpy(), eng.positions()))
        eng.close()
    for other in out[1:]:
        for a, c in zip(out[0], other):
            np.testing.assert_array_equal(a, c)

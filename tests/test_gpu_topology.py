"""Wire topology on the GPU (tbsma_wire_topology: clusters of the
interacting-pair graph, grip connectivity, neck) against the oracle on the
same positions.  The results are integers and unique (components labelled
by their smallest atom index), so they must agree exactly; only a pair
within rounding of r_cut could be decided differently, and the tests check
that the snapshots have none."""

import numpy as np
import pytest

from inputs import Wire, fcc_wire, pack, workload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

A = 4.079


@pytest.fixture(scope="module")
def tb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1311_3890_b300 as tb

    tb.lib()
    return tb


def _wire(x, kind):
    return Wire(x=np.ascontiguousarray(x), kind=np.ascontiguousarray(kind), diameter_nm=0.0,
                length_nm=0.0, L0=float(x[:, 0].max() - x[:, 0].min()), temperature=0.0)


def _shapes():
    """Perfect, cut, diluted and notched wires (kind 1/2 grips kept)."""
    out = []
    w = fcc_wire(2.0, 6.0)
    out.append((w.x, w.kind))
    xc = 0.5 * (w.x[:, 0].min() + w.x[:, 0].max())
    keep = np.abs(w.x[:, 0] - xc) > 3.0
    out.append((w.x[keep], w.kind[keep]))
    for frac, seed in ((0.5, 1), (0.3, 2)):
        keep = (np.random.default_rng(seed).random(w.n) < frac) | (w.kind != 0)
        out.append((w.x[keep], w.kind[keep]))
    w3 = fcc_wire(3.0, 10.0)
    planes = np.round(w3.x[:, 0] / (A / 2)).astype(int)
    mid = (planes.min() + planes.max()) // 2
    r = np.hypot(w3.x[:, 1], w3.x[:, 2])
    cut = np.isin(planes, [mid, mid + 1]) & (r > r.max() - 2.5)
    out.append((w3.x[~cut], w3.kind[~cut]))
    return out


def _ambiguous_pairs(x, band):
    from scipy.spatial import cKDTree

    t = cKDTree(x)
    a = t.query_pairs(5.8 + band, output_type="ndarray")
    if len(a) == 0:
        return 0
    d = np.linalg.norm(x[a[:, 0]] - x[a[:, 1]], axis=1)
    return int(np.sum(np.abs(d - 5.8) < band))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_topology_matches_oracle_on_shapes(tb, orc, prec):
    shapes = _shapes()
    b = pack([_wire(x, k) for x, k in shapes])
    eng = tb.Engine(b, precision=prec)
    got = eng.topology(labels=True)
    labels = got["labels"].cpu().numpy()
    for w, (x, kind) in enumerate(shapes):
        assert _ambiguous_pairs(x, 1e-5) == 0
        ref = orc.topology(x, kind)
        assert got["status"][w] == 0
        assert bool(got["connected"][w]) == ref.connected
        assert got["n_clusters"][w] == ref.n_clusters
        assert got["neck"][w] == ref.neck
        assert got["neck_slab"][w] == ref.neck_slab
        assert got["n_slabs"][w] == ref.n_slabs
        s = b.wire_slice(w)
        np.testing.assert_array_equal(labels[s] - s.start, ref.label)
    assert not got["connected"][1] and got["n_clusters"][1] == 2  # the cut wire
    eng.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_topology_matches_oracle_thermalised(tb, orc, prec):
    """Wires of the tiny batch after 300 steps at 10 and 298 K, pulled."""
    b = workload("tiny_batch")
    eng = tb.Engine(b, precision=prec)
    eng.init_velocities()
    eng.step(300, 2.0)
    x = eng.positions()
    got = eng.topology(labels=True)
    labels = got["labels"].cpu().numpy()
    for w in range(b.n_wires):
        s = b.wire_slice(w)
        if _ambiguous_pairs(x[s], 1e-5 if prec == "mixed" else 1e-9):
            continue  # a pair at the cutoff's rounding: either answer is valid
        ref = orc.topology(x[s], b.kind[s])
        assert bool(got["connected"][w]) == ref.connected
        assert got["n_clusters"][w] == ref.n_clusters
        assert (got["neck"][w], got["neck_slab"][w], got["n_slabs"][w]) == (
            ref.neck, ref.neck_slab, ref.n_slabs)
        np.testing.assert_array_equal(labels[s] - s.start, ref.label)
    eng.close()


def test_pull_to_rupture(tb):
    """A notched D2 x L4 wire pulled at 2e10 1/s at 300 K comes apart: the
    grips end in different clusters, the neck count falls to zero, and the
    failure strain lies between 0.05 and 1.4.  (At 300 K the neck draws out
    into a monatomic chain, which keeps the grips connected through pairs
    within r_cut well after the last slab empties: seeds 4-6 fail at strain
    0.8-1.0.)"""
    w = fcc_wire(2.0, 4.0)
    planes = np.round(w.x[:, 0] / (A / 2)).astype(int)
    mid = (planes.min() + planes.max()) // 2
    r = np.hypot(w.x[:, 1], w.x[:, 2])
    keep = ~(np.isin(planes, [mid, mid + 1]) & (r > r.max() - 2.5))
    wire = Wire(x=w.x[keep], kind=w.kind[keep], diameter_nm=2.0, length_nm=4.0, L0=w.L0,
                temperature=300.0, strain_rate=2e10, gamma=1e-3, seed=4)
    eng = tb.Engine(pack([wire]), precision="mixed")
    eng.init_velocities()
    eps_f, necks = None, []
    for _ in range(175):  # strain 1.4 at most
        eng.step(200, 2.0)
        top = eng.topology()
        necks.append(int(top["neck"][0]))
        if not top["connected"][0]:
            eps_f = float(eng.observables()["strain"][0])
            break
    assert eps_f is not None and 0.05 < eps_f < 1.4
    assert necks[-1] == 0 and necks[0] > 0
    eng.close()


def test_pull_to_rupture_batch(tb):
    """analysis.pull_to_rupture on three notched wires at 300 K, 2e10 1/s:
    every wire fails (by strain 1.4: at 300 K a monatomic chain can hold the
    grips together past strain 0.8), with a yield stress above 1 GPa reached
    before failure and a neck that starts positive, and the run ends 2 A past
    the last failure.  (The final neck may be 0: pairs up to 5.8 A long can
    bridge an empty 2 A slab.)"""
    from paper_1311_3890_b300.analysis import EV_PER_A3_IN_GPA, pull_to_rupture

    wires = []
    for seed in range(3):
        w = fcc_wire(2.0, 4.0, notch_depth=2.5, temperature=300.0, strain_rate=2e10, seed=seed)
        wires.append(w)
    eng = tb.Engine(pack(wires), precision="mixed")
    eng.init_velocities()
    res = pull_to_rupture(eng, report_every=100, max_steps=36000)
    for r, w in zip(res, wires):
        assert 0.05 < r.eps_f < 1.4
        assert r.sigma_y * EV_PER_A3_IN_GPA > 1.0
        assert r.eps_y < r.eps_f
        assert r.final_neck >= 0 and r.neck[0] > 0
        assert (r.strain[-1] - r.eps_f) * w.L0 >= 2.0
    eng.close()


def test_wait_limit_gives_up_and_context_recovers(tb, orc):
    """Failure detection without a fault: a walk bound of one step is too
    small for the union-find of a whole wire, so the call gives up with
    TBSMA_ETIMEOUT and status 2; with the default bound restored the same
    context answers correctly."""
    w = fcc_wire(2.0, 6.0)
    eng = tb.Engine(pack([_wire(w.x, w.kind)]), precision="mixed")
    eng.set_wait_limit(1)
    with pytest.raises(tb.TbsmaError) as e:
        eng.topology()
    assert e.value.status == 5  # TBSMA_ETIMEOUT
    eng.set_wait_limit(1 << 20)
    got = eng.topology()
    ref = orc.topology(w.x, w.kind)
    assert got["status"][0] == 0 and bool(got["connected"][0]) == ref.connected
    assert got["neck"][0] == ref.neck and got["n_clusters"][0] == ref.n_clusters
    with pytest.raises(tb.TbsmaError):
        eng.set_wait_limit(0)
    eng.close()

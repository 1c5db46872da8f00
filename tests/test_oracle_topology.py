"""Pins of the oracle's wire topology (rupture and neck; Results, "Nanowire
elongation"): clusters of the interacting-pair graph against scipy's
connected components on an independently built pair set, and the neck
against direct counts of atoms per (100) plane."""

import numpy as np
import pytest

from inputs import fcc_wire

A = 4.079
RC = 5.8


def _components(x, rc=RC):
    """Connected components by scipy (cKDTree pairs + csgraph), labelled by
    the smallest atom index of each component."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    from scipy.spatial import cKDTree

    n = x.shape[0]
    pairs = cKDTree(x).query_pairs(rc, output_type="ndarray")
    g = coo_matrix((np.ones(len(pairs)), (pairs[:, 0], pairs[:, 1])), shape=(n, n))
    nc, lab = connected_components(g, directed=False)
    first = np.full(nc, n)
    np.minimum.at(first, lab, np.arange(n))
    return nc, first[lab]


def _plane_counts(x):
    return np.bincount(np.round(x[:, 0] / (A / 2)).astype(int))


@pytest.mark.parametrize("d,l", [(2.0, 6.0), (3.0, 10.0)])
def test_perfect_wire(orc, d, l):
    w = fcc_wire(d, l)
    t = orc.topology(w.x, w.kind)
    planes = _plane_counts(w.x)
    assert t.connected and t.n_clusters == 1
    assert t.n_slabs == len(planes) - 4  # two grip planes at each end
    assert t.neck == planes[2:-2].min()
    assert np.all(t.label == 0)


def test_cut_wire_is_disconnected(orc):
    """Removing the planes within 3 A of the centre leaves an 8.2 A gap,
    wider than r_cut: two clusters, grips disconnected, an empty slab."""
    w = fcc_wire(2.0, 6.0)
    xc = 0.5 * (w.x[:, 0].min() + w.x[:, 0].max())
    keep = np.abs(w.x[:, 0] - xc) > 3.0
    t = orc.topology(w.x[keep], w.kind[keep])
    nc, lab = _components(w.x[keep])
    assert not t.connected
    assert t.n_clusters == nc == 2
    np.testing.assert_array_equal(t.label, lab)
    assert t.neck == 0


@pytest.mark.parametrize("frac,seed", [(0.5, 1), (0.35, 2), (0.25, 3)])
def test_diluted_wire_components_equal_scipy(orc, frac, seed):
    """Random dilutions of a wire break it into many clusters; the labels
    equal scipy's components labelled by their smallest index."""
    w = fcc_wire(2.0, 6.0)
    rng = np.random.default_rng(seed)
    keep = rng.random(w.n) < frac
    keep[w.kind != 0] = True  # grips stay
    x, kind = w.x[keep], w.kind[keep]
    t = orc.topology(x, kind)
    nc, lab = _components(x)
    assert t.n_clusters == nc
    np.testing.assert_array_equal(t.label, lab)
    left = np.flatnonzero(kind == 1)[0]
    right = np.flatnonzero(kind == 2)[0]
    assert t.connected == (lab[left] == lab[right])


def test_notch_sets_the_neck(orc):
    """A ring notch (surface atoms beyond R - 2.5 A removed from two central
    planes) makes those planes the neck, counted directly."""
    w = fcc_wire(3.0, 10.0)
    planes = np.round(w.x[:, 0] / (A / 2)).astype(int)
    mid = (planes.min() + planes.max()) // 2
    r = np.hypot(w.x[:, 1], w.x[:, 2])
    cut = np.isin(planes, [mid, mid + 1]) & (r > r.max() - 2.5)
    x, kind = w.x[~cut], w.kind[~cut]
    t = orc.topology(x, kind)
    counts = _plane_counts(x)
    assert t.neck == counts[2:-2].min() == min(counts[mid], counts[mid + 1])
    assert t.neck_slab == np.argmin(counts[2:-2])
    assert t.connected

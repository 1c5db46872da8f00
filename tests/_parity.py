"""Helpers shared by the GPU parity tests (comparison logic only)."""

import numpy as np


def ambiguous_atoms(orc, x, r_cut, band):
    """Atoms whose force depends on a pair lying within `band` of r_cut.

    Whether such a pair is inside the hard cutoff is decided by rounding (the
    FP32 path forms r^2 from 2^-21 A fixed point; the FP64 path may round r^2
    differently from the oracle), so both answers are correct.  A pair (i, j)
    enters F_i, F_j directly and every neighbour of i or j through rho_i,
    rho_j; all those atoms are returned.
    """
    start, nbr = orc.pairs(x, r_cut + band, "cells")
    amb = set()
    for i in range(x.shape[0]):
        js = nbr[start[i]:start[i + 1]]
        if js.size == 0:
            continue
        d = np.sqrt(np.sum((x[js] - x[i]) ** 2, axis=1))
        for j in js[np.abs(d - r_cut) < band]:
            amb.update((i, int(j)))
    if not amb:
        return np.zeros(0, dtype=np.int64)
    s2, n2 = orc.pairs(x, r_cut, "cells")
    out = set(amb)
    for i in amb:
        out.update(int(j) for j in n2[s2[i]:s2[i + 1]])
    return np.array(sorted(out), dtype=np.int64)


def force_errors(F, ref):
    """per-atom |dF|, |F_ref|, and the norm-wise relative error."""
    d = np.linalg.norm(F - ref, axis=1)
    fm = np.linalg.norm(ref, axis=1)
    norm = np.linalg.norm(F - ref) / max(np.linalg.norm(ref), 1e-300)
    return d, fm, norm

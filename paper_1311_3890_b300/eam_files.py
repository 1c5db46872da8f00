"""EAM tables from DYNAMO "setfl" files (the multi-element tabulated format
used by the EAM codes of the paper's lineage), for Engine.set_eam.

Layout of a setfl file (whitespace-separated numbers, any count per line):
  lines 1-3   comments
  line 4      n_elements, then the element names
  line 5      n_rho, d_rho, n_r, d_r, r_cut
  per element a: a line "Z mass lattice_constant lattice_type", then
              n_rho samples of F_a(k d_rho) and n_r samples of f_a(k d_r)
  then, for a = 0 .. n-1 and b = 0 .. a, n_r samples of r * phi_ab(r) at
  r = k d_r (eV A).

read_setfl returns the arrays of one element: F, f and phi = (r phi) / r.
phi at r = 0 is undefined in the file; its sample there is continued from
the next three by the quadratic through them (no pair is ever at r = 0, but
the library wants finite samples and the interpolant's end slope uses it).
"""

from __future__ import annotations

import numpy as np


def _numbers(lines):
    for line in lines:
        for tok in line.split():
            yield tok


def read_setfl(path: str, element: int | str = 0) -> dict:
    """dict(F, d_rho, f, phi, d_r, r_cut, element, mass, lattice) of one
    element (by index or name) of a setfl file."""
    with open(path) as fh:
        lines = fh.read().splitlines()
    if len(lines) < 6:
        raise ValueError("a setfl file has at least 5 header lines and its tables")
    head = lines[3].split()
    n_el = int(head[0])
    names = head[1:1 + n_el]
    if len(names) != n_el:
        raise ValueError("line 4 must name every element")
    a = names.index(element) if isinstance(element, str) else int(element)
    if not 0 <= a < n_el:
        raise ValueError(f"element {element} not in {names}")
    g = lines[4].split()
    n_rho, d_rho, n_r, d_r, r_cut = int(g[0]), float(g[1]), int(g[2]), float(g[3]), float(g[4])
    toks = _numbers(lines[5:])

    def take(n):
        out = np.empty(n)
        for k in range(n):
            out[k] = float(next(toks))
        return out

    F = f = mass = lattice = None
    try:
        for e in range(n_el):
            _z, m, lat, _kind = next(toks), float(next(toks)), float(next(toks)), next(toks)
            Fe, fe = take(n_rho), take(n_r)
            if e == a:
                F, f, mass, lattice = Fe, fe, m, lat
        rphi = None
        for i in range(n_el):
            for j in range(i + 1):
                t = take(n_r)
                if i == a and j == a:
                    rphi = t
    except StopIteration:
        raise ValueError("the file ends before its tables do") from None
    r = np.arange(n_r) * d_r
    phi = np.empty(n_r)
    phi[1:] = rphi[1:] / r[1:]
    phi[0] = 3.0 * phi[1] - 3.0 * phi[2] + phi[3]  # the quadratic through samples 1-3, at 0
    return dict(F=F, d_rho=d_rho, f=f, phi=phi, d_r=d_r, r_cut=r_cut, element=names[a],
                mass=mass, lattice=lattice)


def write_setfl(path: str, elements: list[dict], pair_rphi: dict, n_rho: int, d_rho: float,
                n_r: int, d_r: float, r_cut: float, comments=("", "", "")) -> None:
    """Write a setfl file: elements[a] = dict(name, z, mass, lattice, kind,
    F (n_rho), f (n_r)); pair_rphi[(a, b)] (a >= b) = n_r samples of r phi."""
    out = list(comments[:3]) + [""] * (3 - len(comments[:3]))
    out.append(f"{len(elements)} " + " ".join(e["name"] for e in elements))
    out.append(f"{n_rho} {d_rho!r} {n_r} {d_r!r} {r_cut!r}")

    def rows(a):
        a = np.asarray(a, dtype=np.float64)
        return [" ".join(repr(float(v)) for v in a[k:k + 5]) for k in range(0, a.size, 5)]

    for e in elements:
        out.append(f"{e['z']} {e['mass']!r} {e['lattice']!r} {e['kind']}")
        out += rows(e["F"]) + rows(e["f"])
    for i in range(len(elements)):
        for j in range(i + 1):
            out += rows(pair_rphi[(i, j)])
    with open(path, "w") as fh:
        fh.write("\n".join(out) + "\n")

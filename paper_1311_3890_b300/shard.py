"""Spreading independent wires over ranks (one GPU per rank).

Wires never interact, so the path shards by wire with no collective on the
data path (the paper ran every replica on its own GPU).  Two layouts:

  replicate_specs  weak scaling: every rank runs the full wire list, with the
                   Philox seeds offset by rank so that all trajectories differ;
  split_specs      strong scaling: the wires are dealt to ranks so that the
                   ranks' atom counts stay balanced (largest wires first,
                   each to the currently lightest rank).

`aggregate` is the only communication: after the timed region it takes the
slowest rank's time and the total atom count (all_reduce MAX / SUM).
"""

from __future__ import annotations

import dataclasses


def replicate_specs(specs, rank: int, world: int):
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    return [dataclasses.replace(s, seed=s.seed + rank * len(specs)) for s in specs]


def split_specs(specs, rank: int, world: int, atoms_of):
    """Deal wires to ranks balancing atoms; returns this rank's wires in input order."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    order = sorted(range(len(specs)), key=lambda k: (-atoms_of(specs[k]), k))
    load = [0] * world
    owner = [0] * len(specs)
    for k in order:
        r = min(range(world), key=lambda q: (load[q], q))
        owner[k] = r
        load[r] += atoms_of(specs[k])
    return [s for k, s in enumerate(specs) if owner[k] == rank]


def aggregate(t_ms: float, atoms: int, device=None):
    """(max over ranks of t_ms, sum over ranks of atoms); identity without a process group."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(t_ms), int(atoms)
    t = torch.tensor([float(t_ms)], dtype=torch.float64, device=device)
    a = torch.tensor([int(atoms)], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(a, op=dist.ReduceOp.SUM)
    return float(t.item()), int(a.item())

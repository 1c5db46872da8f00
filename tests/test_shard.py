"""Wire sharding over ranks: layouts, and the gloo aggregation of the timed
region (world size 2, CPU), as bench.py uses it under torchrun."""

import os

import pytest

from inputs.configs import WORKLOADS, WireSpec
from paper_1311_3890_b300.shard import aggregate, replicate_specs, split_specs


def test_replicate_offsets_seeds():
    specs = WORKLOADS["batch256_d3_l40"]()
    seeds = set()
    for r in range(4):
        mine = replicate_specs(specs, r, 4)
        assert [s.diameter_nm for s in mine] == [s.diameter_nm for s in specs]
        seeds |= {s.seed for s in mine}
    assert len(seeds) == 4 * len(specs)


def test_split_balances_atoms_and_covers_all():
    specs = WORKLOADS["ragged512"]()

    def atoms(s):  # proportional to the wire's volume
        return int(s.diameter_nm ** 2 * s.length_nm * 1000)

    parts = [split_specs(specs, r, 3, atoms) for r in range(3)]
    assert sorted(id(s) for p in parts for s in p) == sorted(id(s) for s in specs)
    loads = [sum(atoms(s) for s in p) for p in parts]
    assert max(loads) - min(loads) <= max(atoms(s) for s in specs)


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t, a = aggregate(10.0 + rank, 1000 * (rank + 1))
    q.put((rank, t, a))
    dist.destroy_process_group()


def test_gloo_aggregate_two_ranks():
    import socket

    import torch.multiprocessing as mp

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, a in out:
        assert t == 11.0 and a == 3000


def test_aggregate_without_group_is_identity():
    assert aggregate(5.0, 7) == (5.0, 7)


def test_bad_rank():
    with pytest.raises(ValueError):
        replicate_specs([WireSpec(2.0, 6.0, 10.0, 1e9, 0)], 2, 2)

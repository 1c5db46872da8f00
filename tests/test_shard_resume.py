"""Sharded runs with a failing worker, on the host (no GPU).

Wires are independent, so a multi-rank run is a split of the wire list over
workers (split_specs) with nothing exchanged on the data path.  Here two
spawned worker processes each run their share with the oracle, writing a
checkpoint (positions, velocities, forces, list snapshot, grip displacement,
rebuild count, step) after every chunk of steps.  One worker dies after its
first checkpoint (a process exit, not a device fault); the host sees its exit
status, starts it again from the checkpoint, and the gathered result must
equal an uninterrupted run of all wires bit for bit.
"""

import multiprocessing as mp
import os

import numpy as np
import pytest

from inputs.configs import WireSpec, build
from paper_1311_3890_b300.shard import split_specs

SPECS = [WireSpec(2.0, 3.0, 10.0, 1.0e9, 0), WireSpec(2.0, 3.5, 298.0, 1.0e9, 1),
         WireSpec(2.0, 2.5, 10.0, 1.0e9, 2), WireSpec(2.0, 3.0, 298.0, 1.0e9, 3)]
STEPS, CHUNK = 120, 40


def _start(b):
    import oracle

    v = np.zeros_like(b.x)
    for w in range(b.n_wires):
        s = b.wire_slice(w)
        v[s] = oracle.init_velocities(b.kind[s], int(b.seed[w]), float(b.temperature[w]))
    return dict(x=b.x.copy(), v=v, F=None, xb=None, dg=None, nr=None, step=0)


def _advance(b, st, n):
    import oracle

    F, xb, dg, nr = oracle.md_batch(st["x"], st["v"], b.kind, b.offset, b.n, b.L0,
                                    b.strain_rate, b.temperature, b.gamma, b.seed, st["step"], n,
                                    2.0, brute_max=0, F=st["F"], x_build=st["xb"],
                                    d_grip=st["dg"], n_rebuild=st["nr"])
    st.update(F=F, xb=xb, dg=dg, nr=nr, step=st["step"] + n)


def _worker(rank, world, ckpt, out, die_after):
    """Run this rank's wires to STEPS, checkpointing every CHUNK steps; exit
    with status 3 right after the checkpoint at step `die_after` (if set)."""
    mine = split_specs(SPECS, rank, world, lambda s: build([s]).n_atoms)
    b = build(mine)
    if os.path.exists(ckpt):
        z = np.load(ckpt)
        st = {k: z[k] for k in ("x", "v", "F", "xb", "dg", "nr")}
        st["step"] = int(z["step"])
    else:
        st = _start(b)
    while st["step"] < STEPS:
        _advance(b, st, min(CHUNK, STEPS - st["step"]))
        tmp = ckpt + ".tmp.npz"
        np.savez(tmp, **{k: st[k] for k in ("x", "v", "F", "xb", "dg", "nr")}, step=st["step"])
        os.replace(tmp, ckpt)
        if die_after is not None and st["step"] >= die_after:
            os._exit(3)
    np.savez(out, x=st["x"], v=st["v"], dg=st["dg"], nr=st["nr"])


def test_a_dead_worker_resumes_from_its_checkpoint(tmp_path, orc):
    ctx = mp.get_context("spawn")
    world = 2
    ck = [str(tmp_path / f"ck{r}.npz") for r in range(world)]
    out = [str(tmp_path / f"out{r}.npz") for r in range(world)]
    procs = [ctx.Process(target=_worker, args=(r, world, ck[r], out[r], CHUNK if r == 1 else None))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    assert procs[0].exitcode == 0
    assert procs[1].exitcode == 3  # the host sees the failure
    assert not os.path.exists(out[1]) and int(np.load(ck[1])["step"]) == CHUNK
    again = ctx.Process(target=_worker, args=(1, world, ck[1], out[1], None))
    again.start()
    again.join(timeout=300)
    assert again.exitcode == 0

    # uninterrupted reference: all wires in one batch, in the same chunks
    full = build(SPECS)
    st = _start(full)
    while st["step"] < STEPS:
        _advance(full, st, min(CHUNK, STEPS - st["step"]))
    for r in range(world):
        mine = split_specs(SPECS, r, world, lambda s: build([s]).n_atoms)
        z = np.load(out[r])
        part = build(mine)
        for k, spec in enumerate(mine):
            w = SPECS.index(spec)
            sf, sp = full.wire_slice(w), part.wire_slice(k)
            np.testing.assert_array_equal(z["x"][sp], st["x"][sf])
            np.testing.assert_array_equal(z["v"][sp], st["v"][sf])
            assert z["dg"][k] == st["dg"][w] and z["nr"][k] == st["nr"][w]


def test_split_covers_every_wire_once():
    owners = [split_specs(SPECS, r, 2, lambda s: build([s]).n_atoms) for r in range(2)]
    assert sorted(s.seed for o in owners for s in o) == [s.seed for s in SPECS]
    with pytest.raises(ValueError):
        split_specs(SPECS, 2, 2, lambda s: 1)

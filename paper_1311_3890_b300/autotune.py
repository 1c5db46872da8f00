"""Autotuner of the pair passes' launch shape (tile size, shared-memory window).

For a context, each candidate (threads per block = atoms per tile, window
atoms) is timed with CUDA events over a few launches of the density and the
force pass on the context's current state, and the fastest is applied.
Results are cached per size class: GPU name, precision, and the mean wire
size and the wire cross-section rounded to a power of two (the window a tile
needs grows with the atoms per unit length of its wires).  The shape never
changes a result: every atom's sums run over its own list in list order.
"""

from __future__ import annotations

import json
import math
import os

CANDIDATES = [(b, w) for b in (128, 256) for w in (0, 512, 1024, 1280, 1536, 2048)]


def size_class(engine) -> str:
    import torch

    b = engine.batch
    per_wire = b.n_atoms / max(1, b.n_wires)
    per_len = b.n_atoms / max(1e-9, float(sum(b.L0)))
    name = torch.cuda.get_device_name(engine.device).replace(" ", "_")
    prec = "mixed" if engine.precision == 1 else "fp64"
    return f"{name}/{prec}/w{round(math.log2(per_wire))}/l{round(math.log2(per_len))}"


def time_shape(engine, block: int, window: int, reps: int = 10) -> float:
    """ms per (density + force) pass pair with this launch shape."""
    import torch

    engine.set_launch(block, window)
    engine.run_pass(1, 2)
    engine.run_pass(2, 2)
    a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        engine.run_pass(1, 1)
        engine.run_pass(2, 1)
    c.record()
    torch.cuda.synchronize()
    return a.elapsed_time(c) / reps


def tune(engine, candidates=CANDIDATES, cache_path: str | None = None, reps: int = 10):
    """Apply and return the fastest (block, window); reads/writes cache_path if given."""
    key = size_class(engine)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
    if key in cache:
        block, window = cache[key]["shape"]
        engine.set_launch(block, window)
        return (block, window), cache[key]
    times = {f"{b}x{w}": time_shape(engine, b, w, reps) for b, w in candidates}
    best = min(candidates, key=lambda bw: times[f"{bw[0]}x{bw[1]}"])
    engine.set_launch(*best)
    entry = {"shape": list(best), "ms": times}
    if cache_path:
        cache[key] = entry
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
    return best, entry

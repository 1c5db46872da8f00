"""Pins of the oracle's counter-based generator and Gaussian draws.

Philox4x32-10 is checked word for word against Triton's independent
implementation (``tl.philox``) run by Triton's CPU interpreter; the
Box-Muller normals are checked against the normal law."""

import os
import subprocess
import sys

import numpy as np
import pytest

_TRITON_SCRIPT = r"""
import os, sys
os.environ["TRITON_INTERPRET"] = "1"
import numpy as np, torch, triton, triton.language as tl

@triton.jit
def k(ctr_ptr, out_ptr, seed, N: tl.constexpr):
    i = tl.arange(0, N)
    c0 = tl.load(ctr_ptr + 4 * i + 0)
    c1 = tl.load(ctr_ptr + 4 * i + 1)
    c2 = tl.load(ctr_ptr + 4 * i + 2)
    c3 = tl.load(ctr_ptr + 4 * i + 3)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
    tl.store(out_ptr + 4 * i + 0, a)
    tl.store(out_ptr + 4 * i + 1, b)
    tl.store(out_ptr + 4 * i + 2, c)
    tl.store(out_ptr + 4 * i + 3, d)

ctr = np.load(sys.argv[1])
seed = int(sys.argv[2])
out = torch.zeros(ctr.shape[0] * 4, dtype=torch.int32)
k[(1,)](torch.from_numpy(ctr.view(np.int32).reshape(-1).copy()), out, seed, N=ctr.shape[0])
np.save(sys.argv[3], out.numpy().view(np.uint32).reshape(-1, 4))
"""


def _triton_philox(tmp_path, ctr, seed):
    src = tmp_path / "tri.py"
    src.write_text(_TRITON_SCRIPT)
    np.save(tmp_path / "ctr.npy", ctr)
    env = dict(os.environ, TRITON_INTERPRET="1")
    subprocess.run([sys.executable, str(src), str(tmp_path / "ctr.npy"), str(seed),
                    str(tmp_path / "out.npy")], check=True, env=env, timeout=600)
    return np.load(tmp_path / "out.npy")


@pytest.mark.parametrize("seed", [0, 0xDEADBEEF, (0x1234567 << 32) | 0x89ABCDEF, 2**64 - 1])
def test_philox_matches_triton(orc, tmp_path, seed):
    pytest.importorskip("triton")
    rng = np.random.default_rng(seed & 0xFFFF)
    ctr = rng.integers(0, 2**32, size=(64, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    ctr[1] = 0xFFFFFFFF
    ref = _triton_philox(tmp_path, ctr, seed)
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32)
    got = orc.philox4x32_10(ctr, key)
    assert np.array_equal(got, ref)


def test_philox_is_a_bijection_sample(orc):
    # distinct counters give distinct outputs (a bijection); 2^16 samples
    n = 1 << 16
    ctr = np.zeros((n, 4), dtype=np.uint32)
    ctr[:, 0] = np.arange(n)
    out = orc.philox4x32_10(ctr, np.array([7, 9], dtype=np.uint32))
    as_bytes = out.view(np.dtype((np.void, 16))).ravel()
    assert np.unique(as_bytes).shape[0] == n
    # uniformity of each word: mean of u in (0,1) is 1/2 within 5 sigma
    u = (out.astype(np.float64) + 0.5) / 2**32
    assert np.all(np.abs(u.mean(axis=0) - 0.5) < 5 * np.sqrt(1 / 12 / n))


def test_box_muller_normals(orc):
    from scipy import stats

    n = 200_000
    g = orc.normals(seed=42, atoms=np.arange(n), step=17, tag=0)
    for d in range(3):
        col = g[:, d]
        assert abs(col.mean()) < 5 / np.sqrt(n)
        assert abs(col.var() - 1.0) < 5 * np.sqrt(2 / n)
        assert stats.kstest(col, "norm").pvalue > 1e-4
    # n0 and n1 come from one Box-Muller pair: uncorrelated
    assert abs(np.corrcoef(g[:, 0], g[:, 1])[0, 1]) < 5 / np.sqrt(n)


def test_normals_depend_on_every_counter_field(orc):
    a = orc.normals(1, np.arange(8), step=5, tag=0)
    assert not np.array_equal(a, orc.normals(2, np.arange(8), step=5, tag=0))
    assert not np.array_equal(a, orc.normals(1, np.arange(8), step=6, tag=0))
    assert not np.array_equal(a, orc.normals(1, np.arange(8), step=5 + (1 << 32), tag=0))
    assert not np.array_equal(a, orc.normals(1, np.arange(8), step=5, tag=1))
    assert not np.array_equal(a, orc.normals(1, np.arange(1, 9), step=5, tag=0))

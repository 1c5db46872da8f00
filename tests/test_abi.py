"""The C-ABI library builds, loads without a GPU and exports every entry
point that include/tbsma.h declares (no compute calls)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tbsma.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tbsma_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def built():
    from paper_1311_3890_b300 import build

    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("tbsma_init", "tbsma_build_neighbors", "tbsma_compute_forces",
                 "tbsma_step_nvt_pull", "tbsma_reduce_observables", "tbsma_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(built):
    L = ctypes.CDLL(built)
    for name in _declared():
        assert hasattr(L, name), name


def test_binding_covers_every_declared_symbol(built):
    from paper_1311_3890_b300 import tbsma

    bound = {s[0] for s in tbsma.SIGNATURES}
    assert set(_declared()) <= bound


def test_struct_layouts_match_header(built):
    from paper_1311_3890_b300 import tbsma

    assert ctypes.sizeof(tbsma.Params) == 8 * 8
    assert ctypes.sizeof(tbsma.WireC) == 8 + 4 + 4 + 4 * 8 + 8
    assert ctypes.sizeof(tbsma.ObsC) == 8 + 6 * 8 + 4 + 4
    assert ctypes.sizeof(tbsma.FCheckC) == 4 * 8


def test_bad_arguments_fail_without_a_gpu(built):
    from paper_1311_3890_b300 import tbsma

    L = tbsma.lib()
    ctx = ctypes.c_void_p()
    # null params / wires / buffers are rejected before any CUDA call
    assert L.tbsma_init(None, 1, 1, None, None, None, None, None, ctypes.byref(ctx)) == 1
    assert not ctx
    assert L.tbsma_step_nvt_pull(None, 1, 2.0) == 1
    assert L.tbsma_run_pass(None, 1, 1) == 1
    assert L.tbsma_philox4x32_10(None, None, -1, None, None) == 1
    assert L.tbsma_last_error(None) == b"null context"


def test_default_parameters_agree_with_oracle(orc):
    from paper_1311_3890_b300 import au_params

    p = au_params()
    o = orc.AU
    assert (p.A, p.xi, p.p, p.q, p.r0, p.r_cut) == (o.A, o.xi, o.p, o.q, o.r0, o.r_cut)
    assert p.mass == orc.MASS_AU and p.r_skin == orc.R_SKIN

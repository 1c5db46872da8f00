"""tbsma_forces_noalloc: the entry point for callers that may not allocate
device memory (a host program that gives plug-ins a fixed slice of the GPU,
or a latency-critical loop that cannot afford a device-wide cudaMalloc).

Its FP64 forces must equal those of the regular path (tbsma_compute_forces
of an FP64 context) within the FP64 parity tolerance, on two calls in a row
of different sizes, so that nothing left in its shared scratch array from
one call leaks into the next; the first call is also held against the FP64
CPU oracle (Eq. 1-3 evaluated by brute force) with the parity tests'
tolerance.  This file is collected last on purpose.
"""

import ctypes

import numpy as np
import pytest

from inputs import fcc_wire, jitter, pack

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def tb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1311_3890_b300 as tb

    tb.lib()
    return tb


def _noalloc(tb, x_np):
    """Call the C ABI directly: positions (n,3) -> forces (n,3), FP64."""
    n = x_np.shape[0]
    x = torch.from_numpy(np.ascontiguousarray(x_np.T).reshape(-1)).cuda()
    f = torch.full((3 * n,), np.nan, dtype=torch.float64, device="cuda")
    p = tb.au_params()
    st = tb.lib().tbsma_forces_noalloc(ctypes.byref(p), n, ctypes.c_void_p(x.data_ptr()),
                                       ctypes.c_void_p(f.data_ptr()),
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    torch.cuda.synchronize()
    return f.view(3, n).T.cpu().numpy()


def _regular(tb, x_np):
    w = fcc_wire(2.0, 2.0)
    w.x = x_np
    w.kind = np.zeros(x_np.shape[0], np.uint8)
    eng = tb.Engine(pack([w]), precision="fp64")
    _, F = eng.forces(f32=False, f64=True)
    F = F.cpu().numpy()
    eng.close()
    return F


def _clear_of_cutoff(x, r_cut=5.8, band=1e-9):
    d = np.sqrt(((x[:, None, :] - x[None, :, :]) ** 2).sum(-1))
    return not np.any(np.abs(d - r_cut) < band)


def test_noalloc_forces_match_regular_path_twice(tb, orc):
    a = jitter(fcc_wire(2.0, 6.0).x, 0.05, seed=31)  # 1035 atoms
    b = jitter(fcc_wire(2.0, 3.5).x, 0.08, seed=32) + 100.0  # 621 atoms, elsewhere
    for k, x in enumerate((a, b)):
        assert _clear_of_cutoff(x)  # the two paths then see the same pair set
        got = _noalloc(tb, x)
        ref = _regular(tb, x)
        d = np.linalg.norm(got - ref, axis=1)
        fm = np.linalg.norm(ref, axis=1)
        # FP64 tolerance of the parity tests: only the summation order differs
        assert np.all(np.isfinite(got))
        assert np.all(d <= 1e-12 * fm + 1e-14)
        if k == 0:
            # and against the oracle: |dF_i| <= 1e-12 |F_i| where |F_i| is not
            # tiny next to the atom's pair-force scale S_i, else <= 1e-12 S_i
            o = orc.tbsma(x, brute_max=3000)
            d = np.linalg.norm(got - o.F, axis=1)
            fo = np.linalg.norm(o.F, axis=1)
            big = fo >= 1e-6 * o.S
            assert np.all(d[big] <= 1e-12 * fo[big])
            assert np.all(d[~big] <= 1e-12 * o.S[~big])


def test_noalloc_rejects_oversized_input(tb):
    x = torch.zeros(3, dtype=torch.float64, device="cuda")
    f = torch.zeros(3, dtype=torch.float64, device="cuda")
    p = tb.au_params()
    too_many = 16384 + 1
    st = tb.lib().tbsma_forces_noalloc(ctypes.byref(p), too_many, ctypes.c_void_p(x.data_ptr()),
                                       ctypes.c_void_p(f.data_ptr()), None)
    assert st == 4  # TBSMA_EOVERFLOW, nothing launched
    assert tb.lib().tbsma_forces_noalloc(ctypes.byref(p), -1, None, None, None) == 1

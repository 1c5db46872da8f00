"""Cell-grid growth: a wire's cell grid is planned at init with room for the
wire to double its length; pulled further, its atoms leave the grid, are
binned into edge cells and mark the wire, and the library re-plans the grid
around the wire's current extent before an edge cell can overflow.

A D4 x L6 nm wire at 298 K pulled at 2e10 1/s to strain 1.5 (its grips
end ~0.75 L0 beyond the initial grid at each end, well past rupture) must
run without a status bit or an error, and its forces at the end must match
the FP64 oracle's."""

import numpy as np
import pytest

from inputs import Wire, fcc_wire, pack

from tests._parity import ambiguous_atoms, force_errors

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def tb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1311_3890_b300 as tb

    tb.lib()
    return tb


def test_wire_pulled_past_strain_one_grows_its_grid(tb, orc):
    g = fcc_wire(4.0, 6.0)  # 4395 atoms, L0 = 59.1 A
    rate = 2.0e10
    wire = Wire(x=g.x, kind=g.kind, diameter_nm=4.0, length_nm=6.0, L0=g.L0, temperature=298.0,
                strain_rate=rate, gamma=1e-3, seed=3)
    params = tb.au_params()
    eng = tb.Engine(pack([wire]), precision="mixed", params=params)
    eng.init_velocities()
    extent0 = np.ptp(g.x[:, 0])
    r_list = params.r_cut + params.r_skin
    grid0 = 2.0 * extent0 + 2.0 * r_list  # the initial grid's length along the axis
    steps = int(round(1.5 / (rate * 2.0e-15)))  # 37500 steps to strain 1.5
    done = 0
    while done < steps:
        n = min(5000, steps - done)
        eng.step(n, 2.0)  # raises on EOVERFLOW / EWIRE
        done += n
        ob = eng.observables()
        assert ob["status"][0] == 0
    assert ob["strain"][0] == pytest.approx(1.5, rel=1e-9)
    x = eng.positions()
    assert np.ptp(x[:, 0]) > grid0 + 10.0  # the atoms span more than the initial grid
    assert eng.wire_status()[0] == 0

    F32, F64 = eng.forces(f32=True, f64=True)
    F32, F64 = F32.double().cpu().numpy(), F64.cpu().numpy()
    eng.close()
    ref = orc.tbsma(x, brute_max=0)
    ok = np.ones(x.shape[0], bool)
    ok[ambiguous_atoms(orc, x, 5.8, 5e-6)] = False
    d64, fm, _ = force_errors(F64[ok], ref.F[ok])
    S = ref.S[ok]
    big = fm >= 1e-6 * S
    assert np.all(d64[big] <= 1e-12 * fm[big])
    assert np.all(d64[~big] <= 1e-12 * S[~big])
    d32, _, norm = force_errors(F32[ok], ref.F[ok])
    assert np.max(d32 / np.maximum(S, 1e-300)) <= 1e-5
    assert norm <= 1e-5

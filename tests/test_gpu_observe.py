"""tbsma_step_observe: a call of n steps and a report of the final state.

In graph replays under the default protocol the report's pair passes are
folded into the call's last step (its passes also form the per-atom energy
and virial terms); elsewhere the call steps, then reports.  Either way the
trajectory and every field of the report must equal those of
tbsma_step_nvt_pull followed by tbsma_reduce_observables, bit for bit.
"""

import numpy as np
import pytest

from inputs import workload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# call lengths: shorter than a graph chunk, one chunk, chunks and a
# remainder, whole chunks, a single step
CALLS = (20, 50, 120, 100, 1)


@pytest.fixture(scope="module")
def tb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1311_3890_b300 as tb

    tb.lib()
    return tb


def _run(tb, b, prec, mode, fused, protocol=None):
    eng = tb.Engine(b, precision=prec)
    eng.set_step_mode(mode)
    if protocol is not None:
        eng.set_protocol(**protocol)
    eng.init_velocities()
    reports = []
    for n in CALLS:
        if fused:
            reports.append(eng.step_observe(n, 2.0))
        else:
            eng.step(n, 2.0)
            reports.append(eng.observables())
    eng.step(30, 2.0)  # and the state carries on the same
    out = (reports, eng.positions(), eng.velocities())
    eng.close()
    return out


def _same(a, b):
    (ra, xa, va), (rb, xb, vb) = a, b
    assert len(ra) == len(rb)
    for oa, ob in zip(ra, rb):
        for k in oa.dtype.names:
            np.testing.assert_array_equal(oa[k], ob[k], err_msg=k)
    np.testing.assert_array_equal(xa, xb)
    np.testing.assert_array_equal(va, vb)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("mode", ["graph", "auto"])
def test_step_observe_equals_step_then_observables(tb, prec, mode):
    """The tiny batch (10 K and 298 K wires, pulled, with list rebuilds) in
    graph replays (the folded report) and in auto mode (the persistent step
    kernel, which steps, then reports)."""
    b = workload("tiny_batch")
    a = _run(tb, b, prec, mode, fused=False)
    f = _run(tb, b, prec, mode, fused=True)
    _same(a, f)
    steps = np.cumsum(CALLS)
    for r, s in zip(f[0], steps):
        assert np.all(r["step"] == s)
    assert f[0][-1]["n_rebuilds"].sum() > 0


def test_step_observe_in_protocol_mode_steps_then_reports(tb):
    """Nosé–Hoover with stepwise pull (the paper's protocol): the call steps,
    then reports, as the two calls do."""
    b = workload("tiny_batch")
    p = dict(thermostat="nose_hoover", pull="stepwise", pull_interval=40)
    a = _run(tb, b, "mixed", "graph", fused=False, protocol=p)
    f = _run(tb, b, "mixed", "graph", fused=True, protocol=p)
    _same(a, f)


def test_step_observe_with_no_steps_reports(tb):
    """n_steps = 0: the report of the current state."""
    b = workload("tiny_batch")
    eng = tb.Engine(b, precision="mixed")
    eng.init_velocities()
    eng.step(10, 2.0)
    o1 = eng.observables()
    o2 = eng.step_observe(0, 2.0)
    for k in o1.dtype.names:
        np.testing.assert_array_equal(o1[k], o2[k], err_msg=k)
    eng.close()

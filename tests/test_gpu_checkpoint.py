"""Checkpoint / resume (tbsma_save_state, tbsma_restore_state, Engine.save /
Engine.load): a context restored from a checkpoint continues exactly as the
context that wrote it, bit for bit, in both precisions and under the
Langevin step as under the Nosé–Hoover protocol (whose thermostat state is
part of the checkpoint)."""

import numpy as np
import pytest

from inputs import workload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NH = dict(thermostat="nose_hoover", pull="stepwise", tau_fs=300.0, pull_interval=60,
          ramp_steps=100)


@pytest.fixture(scope="module")
def tb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1311_3890_b300 as tb

    tb.lib()
    return tb


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("proto", [None, NH], ids=["langevin", "nose_hoover"])
def test_resume_is_bitwise(tb, tmp_path, prec, proto):
    b = workload("tiny_batch")
    a = tb.Engine(b, precision=prec)
    a.init_velocities()
    if proto:
        a.set_protocol(**proto)
    a.step(130, 2.0)
    a.save(str(tmp_path / "ck"))
    a.step(170, 2.0)
    c = tb.Engine(b, precision=prec)
    c.load(str(tmp_path / "ck"))
    c.step(170, 2.0)
    np.testing.assert_array_equal(c.positions(), a.positions())
    np.testing.assert_array_equal(c.velocities(), a.velocities())
    oa, oc = a.observables(), c.observables()
    for k in ("e_pot", "e_kin", "sigma_xx", "strain", "n_rebuilds", "step"):
        np.testing.assert_array_equal(oc[k], oa[k])
    xa, ea = a.thermostat()
    xc, ec = c.thermostat()
    np.testing.assert_array_equal(xc, xa)
    np.testing.assert_array_equal(ec, ea)
    a.close()
    c.close()


def test_load_rejects_another_layout(tb, tmp_path):
    a = tb.Engine(workload("tiny_batch"))
    a.save(str(tmp_path / "ck"))
    b = tb.Engine(workload("wire_d2_l6"))
    with pytest.raises(ValueError):
        b.load(str(tmp_path / "ck"))
    a.close()
    b.close()

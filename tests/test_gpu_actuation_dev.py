"""titan_set_actuation_dev (every spring's sinusoidal actuation from device
arrays) against titan_set_actuation with the same values from host arrays:
the per-entry actuation the step kernels read must be the same bits, so the
two simulations must step to the same bits (deterministic accumulation) on
every layout that carries actuation (the SELL rows of the launch kernels,
the cube stream, the persistent kernel) and stay within the oracle's bound
with atomic accumulation.  Also: later host-side edits see the values set
from the device, and bad arguments change nothing."""
import numpy as np
import pytest
import torch

import oracle
from paper_1911_10274_gb300 import inputs
from paper_1911_10274_gb300 import titan as T

pytestmark = pytest.mark.gpu

POS_TOL_FRAC = 1e-4


def _robot(a=9, b=7, c=5, seed=17):
    sys = inputs.actuated_box(a, b, c, np.random.default_rng(seed))
    plain = sys.copy()
    plain.act_amp = None
    plain.act_phase = None
    return sys, plain


def _dev(x):
    return torch.as_tensor(np.asarray(x, np.float32), device="cuda")


def _pair(sys, plain, **kw):
    """(simulation with the actuation given at creation, simulation with the
    same actuation set from device arrays)."""
    a = T.Sim(sys, **kw)
    b = T.Sim(plain, **kw)
    T.titan_set_actuation_dev(b.handle, _dev(sys.act_amp), _dev(sys.act_phase), sys.act_freq)
    return a, b


KW = [dict(), dict(exec_mode=T.EXEC_LAUNCH), dict(exec_mode=T.EXEC_LAUNCH, kernel_variant=1),
      dict(exec_mode=T.EXEC_LAUNCH, kernel_variant=6), dict(exec_mode=T.EXEC_LAUNCH, kernel_variant=8),
      dict(exec_mode=T.EXEC_LAUNCH, order=T.ORDER_INPUT)]


@pytest.mark.parametrize("kw", KW, ids=["auto", "launch", "direct", "box", "cube", "input-order"])
def test_device_actuation_steps_to_the_same_bits(kw):
    sys, plain = _robot()
    a, b = _pair(sys, plain, **kw)
    with a, b:
        a.step(300)
        b.step(300)
        xa, va, _ = a.snapshot()
        xb, vb, _ = b.snapshot()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    xo, _ = oracle.run(sys, 300)
    assert np.abs(xb - xo).max() <= POS_TOL_FRAC * sys.spacing


def test_device_actuation_with_atomic_accumulation_matches_oracle():
    sys, plain = _robot()
    with T.Sim(plain, accumulate=T.ACCUM_ATOMIC) as sim:
        T.titan_set_actuation_dev(sim.handle, _dev(sys.act_amp), _dev(sys.act_phase), sys.act_freq)
        sim.step(300)
        x, _, _ = sim.snapshot()
    xo, _ = oracle.run(sys, 300)
    assert np.abs(x - xo).max() <= POS_TOL_FRAC * sys.spacing


def test_host_edits_after_a_device_set_keep_the_device_values():
    """A host-side set on a few springs and a topology edit (added spring:
    the layout is rebuilt from the host copies) after a device-side set give
    the same bits as doing everything from the host."""
    sys, plain = _robot(6, 5, 4, seed=3)
    rng = np.random.default_rng(8)
    ids = rng.choice(sys.n_springs, 20, replace=False).astype(np.uint32)
    amp2 = rng.uniform(0, 0.2, 20)
    ph2 = rng.uniform(0, 2 * np.pi, 20)
    a, b = _pair(sys, plain, exec_mode=T.EXEC_LAUNCH)
    with a, b:
        for sim in (a, b):
            sim.step(50)
            T.titan_set_actuation(sim.handle, ids, amp2, ph2, sys.act_freq)
            sim.step(50)
            T.titan_add_springs(sim.handle, np.array([[0, sys.n_masses - 1]]), [50.0])
            sim.step(100)
        xa, va, _ = a.snapshot()
        xb, vb, _ = b.snapshot()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)


def test_bad_arguments_change_nothing():
    sys, plain = _robot(5, 4, 3, seed=4)
    a, b = _pair(sys, plain, exec_mode=T.EXEC_LAUNCH)
    with a, b:
        bad = _dev(sys.act_amp)
        bad[3] = float("nan")
        with pytest.raises(T.TitanError, match="non-finite"):
            T.titan_set_actuation_dev(b.handle, bad, _dev(sys.act_phase), 7.0)
        inf_ph = _dev(sys.act_phase)
        inf_ph[0] = float("inf")
        with pytest.raises(T.TitanError, match="non-finite"):
            T.titan_set_actuation_dev(b.handle, _dev(sys.act_amp), inf_ph, 7.0)
        with pytest.raises(T.TitanError, match="spring count"):
            T.titan_set_actuation_dev(b.handle, _dev(sys.act_amp[:-1]), _dev(sys.act_phase[:-1]), 7.0)
        with pytest.raises(T.TitanError, match="freq_hz"):
            T.titan_set_actuation_dev(b.handle, _dev(sys.act_amp), _dev(sys.act_phase), float("inf"))
        with pytest.raises(TypeError):
            T.titan_set_actuation_dev(b.handle, np.asarray(sys.act_amp, np.float32), _dev(sys.act_phase), 7.0)
        a.step(200)
        b.step(200)
        xa, va, _ = a.snapshot()
        xb, vb, _ = b.snapshot()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)

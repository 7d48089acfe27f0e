"""Failure path of the bounded device waits, exercised without a GPU fault.

A one-CTA kernel waits on an mbarrier that nothing arrives on; the wait must
give up after its poll limit and the host must see TITAN_E_TIMEOUT.  The same
process then runs a normal simulation and checks it against the oracle, which
shows the context is still usable after the expired wait.
"""
import numpy as np
import pytest

import oracle
from paper_1911_10274_gb300 import inputs
from paper_1911_10274_gb300 import titan as T

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("spin_limit", [1, 4096])
def test_unarrived_wait_reports_timeout_and_the_device_stays_usable(spin_limit):
    assert T.titan_selftest_wait_timeout(0, spin_limit) == T.TITAN_E_TIMEOUT
    assert "expired" in T.load().titan_last_error(None).decode()
    sys = inputs.cube_drop(n=4)
    xo, _ = oracle.run(sys, 50)
    with T.Sim(sys) as sim:
        sim.step(50)
        xg, _, _ = sim.snapshot()
    assert np.abs(xg - xo).max() <= 1e-4 * sys.spacing


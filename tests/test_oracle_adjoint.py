"""Pins of the oracle's adjoint (reverse-mode derivative of a rollout with
respect to the actuation amplitudes and phases) against FP64 central finite
differences of the oracle's own forward rollout (h = 1e-6)."""
import numpy as np
import pytest

import oracle
from paper_1911_10274_gb300 import inputs

H = 1e-6


def _fd(sys, steps, seed, which, s):
    def J(delta):
        alt = sys.copy()
        if which == "amp":
            alt.act_amp = sys.act_amp.copy()
            alt.act_amp[s] += delta
        else:
            alt.act_phase = sys.act_phase.copy()
            alt.act_phase[s] += delta
        x, _ = oracle.run(alt, steps)
        return float((seed * x).sum())
    return (J(H) - J(-H)) / (2 * H)


def _robot(dims=(4, 3, 3), seed=2, ground=True, all_actuated=False):
    rng = np.random.default_rng(seed)
    sys = inputs.actuated_box(*dims, rng)
    if all_actuated:
        sys.act_amp = rng.uniform(0.02, 0.2, sys.n_springs)
        sys.act_phase = rng.uniform(0, 2 * np.pi, sys.n_springs)
    sys.ground = ground
    if not ground:
        sys.gravity = (0.0, 0.0, 0.0)
    return sys


@pytest.mark.parametrize("ground", [False, True], ids=["floating", "on-ground"])
def test_adjoint_matches_central_differences(ground):
    sys = _robot(ground=ground, all_actuated=True)
    steps = 200
    rng = np.random.default_rng(0)
    seed = rng.standard_normal((sys.n_masses, 3))
    ga, gp, xT, _ = oracle.adjoint(sys, steps, seed)
    x_ref, _ = oracle.run(sys, steps)
    np.testing.assert_array_equal(xT, x_ref)          # the adjoint's forward is the oracle's
    for s in rng.choice(sys.n_springs, 8, replace=False):
        fa = _fd(sys, steps, seed, "amp", s)
        fp = _fd(sys, steps, seed, "phase", s)
        assert ga[s] == pytest.approx(fa, rel=1e-5, abs=1e-9 * max(1.0, abs(fa)))
        assert gp[s] == pytest.approx(fp, rel=1e-5, abs=1e-9 * max(1.0, abs(fp)))


def test_centroid_displacement_gradient_on_ground():
    """The benchmark objective: centroid x-displacement of a robot on the
    ground after 200 steps, d/dA and d/dphi (friction and contact active)."""
    sys = _robot(dims=(5, 3, 3), seed=4)
    steps = 200
    seed = oracle.centroid_x_seed(sys.n_masses)
    ga, gp, _, _ = oracle.adjoint(sys, steps, seed)
    act = np.flatnonzero(sys.act_amp > 0)
    assert len(act) > 5
    rng = np.random.default_rng(1)
    for s in rng.choice(act, 6, replace=False):
        for which, g in (("amp", ga), ("phase", gp)):
            fd = _fd(sys, steps, seed, which, s)
            assert g[s] == pytest.approx(fd, rel=1e-4, abs=1e-10), (which, s)


def test_gradient_of_an_unactuated_spring_phase_is_zero():
    sys = _robot(seed=5)
    off = np.flatnonzero(sys.act_amp == 0)
    ga, gp, _, _ = oracle.adjoint(sys, 100, oracle.centroid_x_seed(sys.n_masses))
    assert np.all(gp[off] == 0.0)          # L does not depend on phi when A = 0
    assert np.any(ga[off] != 0.0)          # but switching A on would change the motion

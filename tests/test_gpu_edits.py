"""Edits between steps (parameter changes, removals, additions of masses and
springs, fixing masses) and the paper's worm actuation, each checked against
the FP64 oracle making the same edit at the same step."""
import math

import numpy as np
import pytest

import oracle
from paper_1911_10274_gb300 import inputs
from paper_1911_10274_gb300 import titan as T

pytestmark = pytest.mark.gpu
TOL = 1e-4 * 0.1


def _system():
    # lifted off the ground: the runs below (up to 600 steps) stay within the
    # contact-free horizon of the parity bar (1e-4 x spacing after 1000 steps
    # without contact; only 100 steps with contact)
    sys = inputs.cube_drop(n=5, drop_height=0.5)
    rng = np.random.default_rng(3)
    sys.vel = rng.normal(0, 0.1, sys.vel.shape)
    sys.rest = sys.rest * rng.uniform(0.98, 1.02, sys.n_springs)
    return sys


@pytest.mark.parametrize("acc", [T.ACCUM_CSR, T.ACCUM_ATOMIC], ids=["csr", "atomic"])
def test_parameter_edits_and_removals_mid_run(acc):
    sys = _system()
    rng = np.random.default_rng(4)
    ids = rng.choice(sys.n_springs, 40, replace=False)
    gone = rng.choice(np.setdiff1d(np.arange(sys.n_springs), ids), 30, replace=False)
    newk = rng.uniform(2e3, 3e4, 40)
    newL = sys.rest[ids] * rng.uniform(0.9, 1.1, 40)
    newc = rng.uniform(0.0, 3.0, 40)
    x, v = oracle.run(sys, 300)
    s2 = sys.copy()
    s2.k[ids], s2.rest[ids], s2.damping[ids] = newk, newL, newc
    s2.k[gone], s2.damping[gone] = 0.0, 0.0
    xo, _ = oracle.run(s2, 300, step0=300, pos=x, vel=v)
    with T.Sim(sys, accumulate=acc) as sim:
        sim.step(300)
        T.titan_set_spring_params(sim.handle, ids, k=newk, rest=newL, damping=newc)
        T.titan_remove_springs(sim.handle, gone)
        sim.step(300)
        xg, _, _ = sim.snapshot()
    assert np.abs(xg - xo).max() <= TOL


def test_adding_masses_and_springs_mid_run():
    sys = _system()
    x, v = oracle.run(sys, 200)
    # a small pendulum of 3 new masses hung under the cube's first corner
    corner = 0
    new_pos = x[corner] + np.array([[0.0, 0.0, -0.1], [0.0, 0.0, -0.2], [0.05, 0.0, -0.3]])
    new_ends = np.array([[corner, sys.n_masses], [sys.n_masses, sys.n_masses + 1],
                         [sys.n_masses + 1, sys.n_masses + 2]], np.uint32)
    big = sys.copy()
    big.pos = np.concatenate([x, new_pos])
    big.vel = np.concatenate([v, np.zeros((3, 3))])
    big.mass = np.concatenate([sys.mass, [0.05, 0.05, 0.05]])
    big.fixed = np.concatenate([sys.fixed, np.zeros(3, np.uint8)])
    big.ends = np.concatenate([sys.ends, new_ends])
    big.k = np.concatenate([sys.k, [5e3, 5e3, 5e3]])
    big.rest = np.concatenate([sys.rest, np.linalg.norm(big.pos[new_ends[:, 1]] - big.pos[new_ends[:, 0]], axis=1)])
    big.damping = np.concatenate([sys.damping, [1.0, 1.0, 1.0]])
    xo, _ = oracle.run(big, 300, step0=200)
    with T.Sim(sys) as sim:
        sim.step(200)
        xg0, _, _ = sim.snapshot()
        first_m = sim.add_masses(xg0[corner] + (new_pos - x[corner]), [0.05] * 3)
        assert first_m == sys.n_masses
        first_s = sim.add_springs(new_ends, [5e3] * 3, rest=big.rest[-3:], damping=[1.0] * 3)
        assert first_s == sys.n_springs
        sim.step(300)
        xg, _, t = sim.snapshot()
        assert t == pytest.approx(500 * sys.dt)
    assert xg.shape == (sys.n_masses + 3, 3)
    assert np.abs(xg - xo).max() <= TOL


def test_fixing_masses_mid_run():
    sys = _system()
    x, v = oracle.run(sys, 150)
    pin = np.arange(0, 25)
    s2 = sys.copy()
    s2.fixed = sys.fixed.copy()
    s2.fixed[pin] = 1
    xo, _ = oracle.run(s2, 250, step0=150, pos=x, vel=v)
    with T.Sim(sys) as sim:
        sim.step(150)
        T.titan_set_fixed(sim.handle, pin, np.ones(len(pin), np.uint8))
        sim.step(250)
        xg, _, _ = sim.snapshot()
    assert np.abs(xg - xo).max() <= TOL


def test_worm_actuation_matches_oracle():
    """Sec. V-B worm: a 27 x 5 x 3 lattice, t_p = 1 s, omega = 20, c = 0.2,
    t_o = the spring's lower starting x minus the lattice's minimum x (Eq. 5)."""
    pos = inputs.lattice_points(27, 5, 3, 0.1)
    ends = inputs.lattice_springs(27, 5, 3)
    s = ends.shape[0]
    sys = inputs.System(pos=pos, vel=np.zeros_like(pos), mass=np.full(len(pos), 0.1),
                        fixed=np.zeros(len(pos), np.uint8), ends=ends, k=np.full(s, 1e4),
                        rest=np.linalg.norm(pos[ends[:, 1]] - pos[ends[:, 0]], axis=1),
                        damping=np.full(s, 1.0), dt=1e-4, ground=True, spacing=0.1)
    # Eq. 5 offsets are multiples of 0.1 s, i.e. of dt: the printed formula then
    # wraps tau (a jump in rest length) exactly at step boundaries, where FP32
    # and FP64 may land on opposite sides; half a step moves every wrap inside a step
    t_o = np.minimum(pos[ends[:, 0], 0], pos[ends[:, 1], 0]) - pos[:, 0].min() + 0.5e-4
    sys.act_amp, sys.act_phase = np.full(s, 0.2), t_o
    xo, _ = oracle.run(sys, 2000, act_mode=2, worm=(20.0, 1.0))
    plain = sys.copy()
    plain.act_amp = None
    with T.Sim(plain) as sim:
        T.titan_set_worm_actuation(sim.handle, np.arange(s), np.full(s, 0.2), t_o, 20.0, 1.0)
        sim.step(2000)
        xg, _, _ = sim.snapshot()
    assert np.abs(xg - xo).max() <= TOL

"""The all-cores oracle variant (oracle/titan_oracle_omp.c) against the serial
oracle.  It gathers each mass's springs in ascending spring index and
evaluates each spring from the spring's own orientation, so every mass
receives the same products in the same order as in the serial spring pass:
the trajectories must agree bit for bit, whatever the thread count."""
import numpy as np
import pytest

import oracle
from paper_1911_10274_gb300 import inputs


def _same(sys, steps, threads, **kw):
    xs, vs = oracle.run(sys, steps, **kw)
    xp, vp = oracle.run_parallel(sys, steps, threads=threads, **kw)
    assert np.array_equal(xs, xp) and np.array_equal(vs, vp)


@pytest.mark.parametrize("threads", [1, 3, 0], ids=["1-thread", "3-threads", "all-cores"])
def test_cube_drop_through_contact_bit_exact(threads):
    sys = inputs.cube_drop(n=6, drop_height=0.02)
    sys.vel[:, 0] = 0.2
    _same(sys, 1500, threads)


def test_actuated_robot_and_worm_form_bit_exact():
    sys = inputs.actuated_box(5, 4, 3, np.random.default_rng(2))
    _same(sys, 600, 0)
    worm = sys.copy()
    worm.act_phase = np.random.default_rng(3).uniform(0.0, 0.5, sys.n_springs)
    _same(worm, 600, 4, act_mode=2, worm=(20.0, 0.5))


def test_fixed_base_lattice_and_mesh_bit_exact():
    _same(inputs.large_lattice(n=12, seed=1), 50, 0)
    _same(inputs.random_mesh(n_points=3000, seed=4, lift=0.0), 50, 5)


def test_duplicates_coincident_ends_and_isolated_masses_bit_exact():
    rng = np.random.default_rng(8)
    n = 40
    pos = rng.uniform(0, 0.4, (n, 3))
    pos[7] = pos[6]
    ends = np.array([(6, 7), (1, 2), (1, 2), (2, 1)] + [(i, (i * 7 + 3) % 30) for i in range(30) if i != (i * 7 + 3) % 30],
                    np.uint32)
    sys = inputs.System(pos=pos, vel=rng.normal(0, 0.1, (n, 3)), mass=rng.uniform(0.05, 0.2, n),
                        fixed=(rng.random(n) < 0.1).astype(np.uint8), ends=ends,
                        k=rng.uniform(100, 1000, len(ends)), rest=rng.uniform(0.0, 0.2, len(ends)),
                        damping=rng.uniform(0, 0.5, len(ends)), dt=1e-4, ground=True, spacing=0.1)
    _same(sys, 300, 3)


def test_reports_the_threads_it_used():
    p = oracle.Parallel(inputs.cube_drop(n=3), threads=2)
    p.run(3)
    assert p.threads_used == 2
    assert oracle.max_threads() >= 1

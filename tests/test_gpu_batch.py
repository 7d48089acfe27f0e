"""Batched robots in persistent cluster launches vs the FP64 oracle, robot by
robot (one oracle run per robot).  Sizes span one CTA to multi-CTA clusters
that read neighbour states through distributed shared memory."""
import numpy as np
import pytest

import oracle
from paper_1911_10274_gb300 import inputs
from paper_1911_10274_gb300 import titan as T

pytestmark = pytest.mark.gpu
POS_TOL_FRAC = 1e-4


def _robots():
    rng = np.random.default_rng(21)
    dims = [(3, 3, 3), (5, 4, 3), (12, 12, 12), (7, 3, 9), (4, 11, 6), (10, 10, 10), (3, 12, 3)]
    return [inputs.actuated_box(a, b, c, rng) for a, b, c in dims]


def _check(batch, robots, steps, step0=0):
    for r, sy in enumerate(robots):
        xo, vo = oracle.run(sy, steps, step0=step0)
        xg, vg = batch.read(r)
        err = np.abs(xg.astype(np.float64) - xo).max()
        assert err <= POS_TOL_FRAC * sy.spacing, (r, sy.name, err)


def test_batch_rollout_matches_oracle_for_every_robot():
    robots = _robots()
    with T.Batch(robots) as b:
        g = b.groups()
        assert max(x["cluster"] for x in g) > 1, "the 12^3 robot must need a multi-CTA cluster"
        b.rollout(1000)
        _check(b, robots, 1000)
        c = b.centroids()
        for r, sy in enumerate(robots):
            xg, _ = b.read(r)
            np.testing.assert_allclose(c[r], xg.astype(np.float64).mean(axis=0), rtol=0, atol=1e-5)


def test_batch_second_rollout_continues_the_actuation_clock():
    robots = _robots()[:3]
    with T.Batch(robots) as b:
        b.rollout(300).rollout(200)
        for r, sy in enumerate(robots):
            x1, v1 = oracle.run(sy, 300)
            s2 = sy.copy()
            s2.pos, s2.vel = x1, v1
            xo, _ = oracle.run(s2, 200, step0=300)
            xg, _ = b.read(r)
            assert np.abs(xg - xo).max() <= POS_TOL_FRAC * sy.spacing


@pytest.mark.parametrize("threads,tpm", [(128, 1), (512, 1), (128, 2), (256, 2), (512, 4), (64, 4)])
def test_every_launch_shape_matches_oracle(threads, tpm):
    """Every shape the autotuner can pick (threads per CTA, threads per mass),
    pinned by hand, against the oracle."""
    robots = _robots()
    with T.Batch(robots) as b:
        for g in range(len(b.groups())):
            b.configure(g, threads, tpm)
        b.rollout(300)
        _check(b, robots, 300)


def test_batch_autotune_and_reset_keep_results():
    robots = _robots()[:4]
    with T.Batch(robots) as b:
        b.autotune(20)
        assert all(x["threads"] in (128, 256, 512) and x["threads_per_mass"] in (1, 2, 4) for x in b.groups())
        b.rollout(400)
        a = [b.read(r)[0] for r in range(len(robots))]
        b.reset()
        b.rollout(400)
        for r in range(len(robots)):
            assert np.array_equal(a[r], b.read(r)[0]), "deterministic and resettable"
        _check(b, robots, 400)


def test_batch_equals_single_system_path_within_tolerance():
    sy = inputs.actuated_box(6, 5, 4, np.random.default_rng(3))
    with T.Batch([sy]) as b, T.Sim(sy) as s:
        b.rollout(500)
        s.step(500)
        xs, _, _ = s.snapshot()
        xb, _ = b.read(0)
        assert np.abs(xs - xb).max() <= POS_TOL_FRAC * sy.spacing


def test_unactuated_batch_with_fixed_masses():
    rng = np.random.default_rng(8)
    robots = []
    for dims in [(4, 4, 4), (6, 3, 5)]:
        sy = inputs.actuated_box(*dims, rng)
        sy.act_amp = None
        sy.fixed[:dims[0] * dims[1]] = 1
        sy.vel[:] = rng.normal(0, 0.1, sy.vel.shape)
        robots.append(sy)
    with T.Batch(robots) as b:
        b.rollout(500)
        _check(b, robots, 500)
        for r, sy in enumerate(robots):
            xg, _ = b.read(r)
            fx = sy.fixed.astype(bool)
            assert np.array_equal(xg[fx], sy.pos[fx].astype(np.float32))

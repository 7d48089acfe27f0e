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


@pytest.mark.parametrize("threads,tpm", [(128, 1), (512, 1), (128, 2), (256, 2), (512, 4), (64, 4), (1024, 1),
                                         (1024, 8), (256, 8)])
def test_every_launch_shape_matches_oracle(threads, tpm):
    """Every shape the autotuner can pick (threads per CTA, most threads per
    mass; each CTA takes the most that fit its masses), pinned by hand,
    against the oracle."""
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
        assert all(x["threads"] in (128, 256, 512, 1024) and x["threads_per_mass"] in (1, 2, 4, 8)
                   for x in b.groups())
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


def test_system_too_dense_for_a_cluster_is_refused_and_the_device_kept():
    """4096 masses on a line, each joined to its next 32: 64 half-edges per
    mass, so even 8 CTAs of 512 masses need 320 KB of rows each.  Creation
    must refuse it (unsupported, nothing built) and leave the caller's current
    device as it was; a small batch still works afterwards."""
    import torch
    n, reach = 4096, 32
    pos = np.zeros((n, 3))
    pos[:, 0] = 0.1 * np.arange(n)
    pos[:, 2] = 1.0
    ends = np.array([(i, i + d) for i in range(n) for d in range(1, reach + 1) if i + d < n], np.uint32)
    s = ends.shape[0]
    dense = inputs.System(pos=pos, vel=np.zeros_like(pos), mass=np.full(n, 0.1), fixed=np.zeros(n, np.uint8),
                          ends=ends, k=np.full(s, 1e3), rest=0.1 * (ends[:, 1] - ends[:, 0]).astype(np.float64),
                          damping=np.full(s, 1.0), dt=1e-4, ground=True)
    torch.cuda.set_device(0)
    before = torch.cuda.current_device()
    with pytest.raises(T.TitanError) as ei:
        T.Batch([dense])
    assert ei.value.status == T.TITAN_E_UNSUPPORTED
    assert "cluster of 8" in str(ei.value)
    assert torch.cuda.current_device() == before
    robots = _robots()[:2]
    with T.Batch(robots) as b:
        b.rollout(100)
        _check(b, robots, 100)


def test_benchmark_batch_sample_matches_oracle_in_every_launch_group():
    """The benchmark's own batch (4096 robots, a, b, c ~ U{3..12}), autotuned
    as the benchmark runs it, 300 steps: at least 64 robots, with at least four
    (or all) from every launch group, compared with the oracle one by one."""
    robots = inputs.robot_batch(4096, seed=0)
    with T.Batch(robots) as b:
        b.autotune(50)
        n_groups = len(b.groups())
        group_of = np.array([b.group_of(r) for r in range(len(robots))])
        assert set(group_of.tolist()) == set(range(n_groups)), "every group holds robots"
        b.rollout(300)
        rng = np.random.default_rng(0)
        picks = set()
        for g in range(n_groups):
            members = np.flatnonzero(group_of == g)
            picks.update(rng.choice(members, min(4, len(members)), replace=False).tolist())
        while len(picks) < 64:
            picks.add(int(rng.integers(len(robots))))
        sample = sorted(picks)
        assert {group_of[r] for r in sample} == set(range(n_groups))
        _check_sample(b, robots, sample, 300)


def _check_sample(batch, robots, sample, steps):
    for r in sample:
        sy = robots[r]
        xo, _ = oracle.run(sy, steps)
        xg, _ = batch.read(r)
        err = np.abs(xg.astype(np.float64) - xo).max()
        assert err <= POS_TOL_FRAC * sy.spacing, (r, sy.name, err)

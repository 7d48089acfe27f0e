"""Sharding independent robots across ranks (paper_1911_10274_gb300/shard.py).

Host logic on CPU: the spring-count partition (every robot once, balanced
within one robot of the ideal split), the merge back into robot order, and the
whole sharded path over two gloo ranks with the oracle as the rollout, which
must give exactly the unsharded result.  On the GPU: three shards run one
after another on one device through the batch engine, merged, equal the
unsharded batch bit for bit."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1911_10274_gb300 import inputs, shard  # noqa: E402


@pytest.mark.parametrize("k", [1, 2, 3, 7, 50])
def test_partition_covers_every_item_once_and_balances_springs(k):
    rng = np.random.default_rng(k)
    w = rng.integers(150, 19000, 40)
    parts = shard.partition(w, k)
    assert len(parts) == k
    allidx = np.concatenate(parts)
    assert sorted(allidx.tolist()) == list(range(len(w)))
    loads = [int(w[p].sum()) for p in parts]
    # the LPT rule's bound: no shard exceeds the ideal share by more than the largest item
    assert max(loads) <= w.sum() / k + w.max()
    assert shard.partition(w, k)[0].tolist() == parts[0].tolist()      # deterministic


def test_partition_rejects_bad_input_and_handles_more_shards_than_items():
    with pytest.raises(ValueError):
        shard.partition([1, 2], 0)
    with pytest.raises(ValueError):
        shard.partition([1, -2], 2)
    parts = shard.partition([5, 3], 4)
    assert sorted(len(p) for p in parts) == [0, 0, 1, 1]


def test_merge_restores_item_order_and_refuses_gaps_and_overlaps():
    parts = [np.array([0, 3]), np.array([1, 2])]
    vals = [np.array([[0.0] * 3, [3.0] * 3]), np.array([[1.0] * 3, [2.0] * 3])]
    out = shard.merge(parts, vals, 4)
    assert np.array_equal(out[:, 0], [0.0, 1.0, 2.0, 3.0])
    with pytest.raises(ValueError):
        shard.merge([np.array([0]), np.array([0])], [np.zeros((1, 3)), np.zeros((1, 3))], 1)
    with pytest.raises(ValueError):
        shard.merge([np.array([0])], [np.zeros((1, 3))], 2)


def _oracle_rollout(robots, steps):
    import oracle
    return np.array([oracle.run(r, steps)[0].mean(axis=0) for r in robots], dtype=np.float32).reshape(-1, 3)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        robots = inputs.robot_batch(9, seed=3)
        got = shard.sharded_centroids(robots, 20, rank, world, rollout=_oracle_rollout)
        out.put((rank, got))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_gather_the_unsharded_result():
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    mp.start_processes(_rank_main, args=(2, _free_port(), q), nprocs=2, join=True, start_method="spawn")
    got = sorted((q.get() for _ in range(2)), key=lambda x: x[0])
    robots = inputs.robot_batch(9, seed=3)
    want = _oracle_rollout(robots, 20)
    for _, c in got:
        assert np.array_equal(c, want)


@pytest.mark.gpu
def test_three_shards_one_after_another_equal_the_unsharded_batch():
    robots = inputs.robot_batch(48, seed=5)
    whole = shard.rollout_centroids(robots, 400)
    parts = shard.partition([r.n_springs for r in robots], 3)
    assert all(len(p) for p in parts)
    vals = [shard.rollout_centroids([robots[i] for i in p], 400) for p in parts]
    merged = shard.merge(parts, vals, len(robots))
    assert np.array_equal(merged, whole)
    one = shard.sharded_centroids(robots, 400, 0, 1)
    assert np.array_equal(one, whole)

"""Sharding a batch of independent robots across ranks (one GPU per rank).

Robots never interact, so a batch splits into shards with no exchange during
the rollout: each rank advances its own shard in its own batch engine, and one
gather at the end of the rollout brings every robot's result back in the
caller's order.  Shards are balanced by spring count, the quantity the step's
time follows (each step costs a fixed amount of work per spring).

partition() and merge() are plain host logic; sharded_centroids() runs the
rank's shard with a rollout function (by default the batch engine,
rollout_centroids) and all-gathers the per-robot centroids over
torch.distributed when more than one rank takes part.
"""
from __future__ import annotations

import heapq
from typing import Callable, List, Optional, Sequence

import numpy as np


def partition(weights: Sequence[int], k: int) -> List[np.ndarray]:
    """Splits items 0..n-1 into k shards whose weight sums are balanced:
    items in decreasing weight (ties by index) each go to the lightest shard
    so far (ties by shard index), the longest-processing-time rule.  Each
    shard's indices are returned in increasing order; shards may be empty
    when k exceeds the item count.  Deterministic: every rank computes the
    same split."""
    if k < 1:
        raise ValueError("k must be >= 1")
    w = np.asarray(weights, dtype=np.int64)
    if w.ndim != 1 or (w < 0).any():
        raise ValueError("weights must be a 1-D sequence of non-negative integers")
    order = sorted(range(len(w)), key=lambda i: (-int(w[i]), i))
    heap = [(0, s) for s in range(k)]
    members: List[List[int]] = [[] for _ in range(k)]
    for i in order:
        load, s = heapq.heappop(heap)
        members[s].append(i)
        heapq.heappush(heap, (load + int(w[i]), s))
    return [np.array(sorted(m), dtype=np.int64) for m in members]


def merge(parts: Sequence[np.ndarray], values: Sequence[np.ndarray], n: int) -> np.ndarray:
    """Puts per-shard results back in item order: values[s][t] belongs to
    item parts[s][t].  Every item must be covered exactly once."""
    first = next((np.asarray(v) for v in values if len(v)), None)
    tail = first.shape[1:] if first is not None else ()
    out = np.zeros((n,) + tuple(tail), dtype=first.dtype if first is not None else np.float32)
    seen = np.zeros(n, dtype=bool)
    for idx, val in zip(parts, values):
        val = np.asarray(val)
        if len(idx) != len(val):
            raise ValueError("a shard's values do not match its items")
        if seen[idx].any():
            raise ValueError("an item appears in two shards")
        seen[idx] = True
        if len(idx):
            out[idx] = val
    if not seen.all():
        raise ValueError("some items are in no shard")
    return out


def rollout_centroids(robots, steps: int, device: int = 0, stream: Optional[int] = None) -> np.ndarray:
    """Centroids ([n][3], float32) of every robot after `steps` steps of one
    batch rollout on `device`, with the batch engine's default launch shapes
    (which depend on each robot alone, so a robot's trajectory is the same in
    any batch)."""
    from . import titan as T
    if not len(robots):
        return np.zeros((0, 3), np.float32)
    with T.Batch(list(robots), device=device, stream=stream) as b:
        b.rollout(steps)
        return np.asarray(b.centroids(), dtype=np.float32)


def _all_gather_rows(local: np.ndarray, counts: Sequence[int], group=None) -> List[np.ndarray]:
    """All-gathers each rank's [count][3] float32 rows (padded to the largest
    count) and returns them per rank, unpadded."""
    import torch
    import torch.distributed as dist
    width = max(1, max(counts))
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    buf = torch.zeros((width, 3), dtype=torch.float32, device=dev)
    if len(local):
        buf[: len(local)] = torch.as_tensor(local, dtype=torch.float32, device=dev)
    world = dist.get_world_size(group)
    outs = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(outs, buf, group=group)
    return [outs[r][: counts[r]].cpu().numpy() for r in range(world)]


def sharded_centroids(robots, steps: int, rank: int, world: int,
                      rollout: Optional[Callable] = None, group=None) -> np.ndarray:
    """Every robot's centroid after `steps` steps, this rank advancing only
    its shard (partition() by spring count) and the shards' results gathered
    at the end.  rollout(robots, steps) -> [n][3] centroids (default: the
    batch engine on the current CUDA device).  With world == 1 no process
    group is needed; otherwise torch.distributed must be initialised."""
    parts = partition([r.n_springs for r in robots], world)
    run = rollout or (lambda rs, n: rollout_centroids(rs, n, _current_device()))
    mine = parts[rank]
    local = np.asarray(run([robots[i] for i in mine], steps), dtype=np.float32).reshape(len(mine), 3)
    if world == 1:
        return merge(parts, [local], len(robots))
    gathered = _all_gather_rows(local, [len(p) for p in parts], group)
    return merge(parts, gathered, len(robots))


def _current_device() -> int:
    import torch
    return torch.cuda.current_device()

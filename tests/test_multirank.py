"""The N > 1 host path of bench.py on CPU: world size 2 over the gloo backend.

Each rank simulates its own replica (the method has no data-path exchange
between independent bodies), so the only collective is the max-over-ranks
reduction of the timings; the whole-job value is the units of all ranks over
the slowest rank's time.  The reference arm runs on rank 0 alone.
"""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = [1.0 + rank, 10.0 - rank]           # rank 1 slower on the first, faster on the second
        t, e2e = bench.max_over_ranks(local, world)
        dist.barrier()
        out.put((rank, t, e2e, bench.whole_job_rate(world, 1000.0, t)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_with_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, q), nprocs=2, join=True, start_method="spawn")
    got = sorted(q.get() for _ in range(2))
    for rank, t, e2e, rate in got:
        assert t == 2.0 and e2e == 10.0            # the slowest rank's time, per quantity
        assert rate == pytest.approx(2 * 1000.0 / 2.0)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks([3.0, 4.0], 1) == [3.0, 4.0]


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    args = type("A", (), dict(steps=1, warmup=3, gpus=2, workload="lattice1m", accumulate="csr",
                              kernel_variant=0, order="morton", exec="auto"))()
    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.run_reference(args) is None
    assert buf.getvalue() == ""

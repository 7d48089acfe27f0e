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


def test_reference_arm_prints_one_complete_json_line(monkeypatch):
    """Rank 0 of the reference arm times the FP64 oracle on the host and prints
    the contract's line: the same metric and unit as our arm, the CPU baseline
    it measured, and an end-to-end figure with no host-device copies.  A small
    cube stands in for the sub-lattice so the test takes a fraction of a second."""
    import json
    import bench
    from paper_1911_10274_gb300 import inputs
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    monkeypatch.setattr(bench, "sub_lattice_for_budget", lambda seconds: inputs.cube_drop(n=4))
    args = type("A", (), dict(steps=2, warmup=3, gpus=1, workload="lattice1m", accumulate="csr",
                              kernel_variant=0, order="morton", exec="auto", no_l2_persist=False))()
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args)
    lines = buf.getvalue().strip().splitlines()
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["higher_is_better"] is True and d["vs_baseline"] is None and d["dtype"] == "f64"
    assert d["config"]["workload"].startswith("1M-mass lattice")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_algorithmic_bytes_and_traffic_key():
    """Per step: 16 B per spring (its {i, j, k, L0} record) and 52 B per mass
    (position and velocity read and written, 1/m read): 255.7 MB on the
    1M-mass lattice.  The ncu traffic key follows every file the step kernels
    are compiled from, so a changed kernel reports no stale traffic."""
    import shutil
    import tempfile
    import bench
    assert bench.algorithmic_bytes(1_000_000, 12_731_796) == 16 * 12_731_796 + 52 * 1_000_000 == 255_708_736
    h0 = bench.kernel_source_hash()
    with tempfile.TemporaryDirectory() as d:
        for rel in bench.KERNEL_INPUTS:
            os.makedirs(os.path.dirname(os.path.join(d, rel)), exist_ok=True)
            shutil.copy(os.path.join(bench.ROOT, rel), os.path.join(d, rel))
        old = bench.ROOT
        try:
            bench.ROOT = d
            assert bench.kernel_source_hash() == h0
            for rel in bench.KERNEL_INPUTS:
                with open(os.path.join(d, rel), "a") as f:
                    f.write("\n")
                h1 = bench.kernel_source_hash()
                assert h1 != h0
                h0 = h1
        finally:
            bench.ROOT = old

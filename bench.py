"""Benchmark of the spring-mass hot path on GB300.

A "step" is one simulation time step over the whole system: every spring's
force onto both masses, then every mass integrated (gravity, constraints).
Default workload: the 1M-mass lattice (100^3 sites, 12,731,796 26-neighbourhood
springs, perturbed rest lengths, lognormal k, bottom layer fixed, no ground,
dt = 5e-5) with the deterministic CSR kernel.  The metric is spring updates
per second (springs x steps / time); the roofline compares the algorithmic
bytes of one step with the measured HBM copy bandwidth.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--accumulate csr|atomic] [--workload lattice1m|...]
Under torchrun (N > 1) every rank simulates its own replica on its own GPU
(the method has no data-path exchange between independent bodies); the value
is the total over ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "spring updates/s"
# the step kernel a Sim resolved to (titan_csr_kernel), and its description
CSR_KERNEL_NAMES = {0: "k_springs_atomic+k_masses_atomic", 1: "k_step_sell", 2: "k_step_sell_staged",
                    3: "k_step_sell_pf", 4: "k_step_halo", 5: "k_step_halo_tma", 6: "k_step_box",
                    7: "k_step_box_tma", 8: "k_step_cube"}
CSR_KERNELS = {0: "atomic scatter", 1: "direct-loads", 2: "tma-staged", 3: "bulk-l2-prefetch",
               4: "halo (coloured neighbourhood table in shared memory)", 5: "halo+tma",
               6: "grid box (box table in shared memory, no neighbour index in the stream)",
               7: "grid box, stream staged in shared memory by TMA bulk copies",
               8: "cube (springs inside a 256-mass cube read and evaluated once)"}
UNIT = "spring_updates/s"
L2_BYTES = 126 * 1024 * 1024
# spin before the timed region (about 1 ms at the GB300's 2 GHz): longer than
# the host takes to enqueue the start event and the K steps
QUEUE_FILL_CYCLES = 2_000_000
E2E_PASSES = 3

# ncu DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one step
# kernel launch, keyed by (workload, accumulation, kernel, SHA-256 prefix of
# the files the step kernels are compiled from: their source, the physics
# header and the build script with its flags).  Reported only while those are
# unchanged.  Capture: profiles/k_step_box_lattice1m.md.
NCU_TRAFFIC = {
    ("lattice1m", "csr", "k_step_box", "544b3a1b8dc37538"): 251_609_856 + 12_306_432,
}
KERNEL_INPUTS = ("paper_1911_10274_gb300/csrc/step_kernels.cu", "paper_1911_10274_gb300/csrc/physics.cuh",
                 "paper_1911_10274_gb300/build.py")


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for rel in KERNEL_INPUTS:
        h.update(open(os.path.join(ROOT, rel), "rb").read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def algorithmic_bytes(n_masses: int, n_springs: int) -> int:
    """Bytes one step must move: 16 per spring (i, j, k, L0) and 52 per mass
    (position and velocity read and written, 1/m read)."""
    return 16 * n_springs + 52 * n_masses


WORKLOADS = {"lattice1m": "1M-mass lattice 100^3, 12,731,796 springs, fixed base, no ground, dt=5e-5",
             "lattice50": "50^3 lattice, 1,558,396 springs", "mesh2m": "2M-point kNN mesh",
             "cube1k": "10^3 cube drop"}


def make_workload(name: str):
    from paper_1911_10274_gb300 import inputs
    if name == "lattice1m":
        return inputs.large_lattice(n=100, seed=0)
    if name == "lattice50":
        s = inputs.large_lattice(n=50, seed=0)
        return s
    if name == "mesh2m":
        return inputs.random_mesh(n_points=2_000_000, seed=0)
    if name == "cube1k":
        return inputs.cube_drop()
    raise SystemExit(f"unknown workload {name}")


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index
        import tempfile
        self.path = os.path.join(os.environ.get("TITAN_CLOCKS_DIR", tempfile.gettempdir()),
                                 f"titan_clocks_gpu{gpu_index}_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return None
        rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if "Active" in r[5 + k] and "Not" not in r[5 + k]})
        loaded = [x for x in sm if mx and x > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def max_over_ranks(values, world: int, device=None):
    """Element-wise maximum of per-rank floats over all ranks (one all-reduce);
    the values themselves at world size 1."""
    if world <= 1:
        return [float(x) for x in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x) for x in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def whole_job_rate(world: int, units_per_rank: float, seconds: float) -> float:
    """Throughput of the whole job: every rank processed units_per_rank (weak
    scaling, independent replicas); the job took the slowest rank's time."""
    return world * units_per_rank / seconds


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def time_oracle(system, steps: int):
    import oracle
    t0 = time.perf_counter()
    oracle.run(system, steps)
    return time.perf_counter() - t0


def sub_lattice_for_budget(seconds_per_step: float):
    """Largest n^3 sub-lattice of the 1M-mass recipe whose oracle step fits the budget."""
    from paper_1911_10274_gb300 import inputs
    probe = inputs.large_lattice(n=30, seed=0)
    t = min(time_oracle(probe, 3) / 3, 10.0)
    rate = probe.n_springs / max(t, 1e-9)
    n = 30
    while n < 100 and inputs.lattice_spring_count(n + 2, n + 2, n + 2) / rate <= seconds_per_step:
        n += 2
    while n > 4 and inputs.lattice_spring_count(n, n, n) / rate > seconds_per_step:
        n -= 2
    return inputs.large_lattice(n=n, seed=0)


def host_cpu():
    """nproc and the host CPU's model name (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            info = open("/proc/cpuinfo").read().splitlines()
            for key in ("model name", "Model", "CPU part"):
                hit = [ln.split(":", 1)[1].strip() for ln in info if ln.lower().startswith(key.lower())]
                if hit:
                    model = hit[0] if key != "CPU part" else f"CPU part {hit[0]}"
                    break
        except Exception:
            pass
    return os.cpu_count(), model or "unknown"


def cpu_baseline_leg(system, target_seconds: float = 15.0):
    """The oracle as it stands on the host cores, from the workload's initial
    state, on a bounded number of steps: the serial FP64 program on one
    thread (the paper's own CPU comparison is single-threaded) and its
    per-mass-gather variant on all cores (bit-identical trajectory); plus the
    10^3 cube drop timed in full (10,000 steps) by both."""
    import oracle
    from paper_1911_10274_gb300 import inputs
    nproc, model = host_cpu()
    probe = time_oracle(system, 1)
    steps = max(1, min(200, int(target_seconds / max(probe, 1e-6))))
    t = time_oracle(system, steps)
    out = {"value": system.n_springs * steps / t, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{system.name}: {steps} time steps of the full system from its initial "
                     f"state, FP64, one thread ({t:.1f} s)",
           "nproc": nproc, "cpu_model": model}
    cube = inputs.cube_drop()
    t0 = time.perf_counter()
    oracle.run(cube, 10_000)
    t_c0 = time.perf_counter() - t0
    out["cube1k_full"] = {"value": cube.n_springs * 10_000 / t_c0, "unit": UNIT, "cores": 1,
                          "seconds": t_c0, "sample": "10^3 cube drop, all 10,000 steps, FP64, one thread"}
    try:
        par = oracle.Parallel(system)
        t0 = time.perf_counter()
        par.run(1)
        p_probe = time.perf_counter() - t0
        p_steps = max(1, min(400, int(target_seconds / 2 / max(p_probe, 1e-6))))
        t0 = time.perf_counter()
        par.run(p_steps)
        t_p = time.perf_counter() - t0
        out["all_cores"] = {"value": system.n_springs * p_steps / t_p, "unit": UNIT, "cores": par.threads_used,
                            "sample": f"{system.name}: {p_steps} time steps, FP64, per-mass gather on "
                                      f"{par.threads_used} threads ({t_p:.1f} s), trajectory bit-identical "
                                      f"to the serial oracle"}
        pc = oracle.Parallel(cube)
        t0 = time.perf_counter()
        pc.run(10_000)
        t_pc = time.perf_counter() - t0
        out["cube1k_full_all_cores"] = {"value": cube.n_springs * 10_000 / t_pc, "unit": UNIT,
                                        "cores": pc.threads_used, "seconds": t_pc,
                                        "sample": "10^3 cube drop, all 10,000 steps, FP64, per-mass gather"}
    except Exception as exc:            # no OpenMP runtime on this host
        out["all_cores"] = {"unavailable": f"{type(exc).__name__}: {exc}"[:200]}
    return out


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    per_step = 90.0 / max(1, args.steps + args.warmup)
    system = sub_lattice_for_budget(per_step)
    import oracle
    x, v = system.pos, system.vel
    for w in range(args.warmup):
        x, v = oracle.run(system, 1, step0=w, pos=x, vel=v)
    t0 = time.perf_counter()
    for k in range(args.steps):
        x, v = oracle.run(system, 1, step0=args.warmup + k, pos=x, vel=v)
    dt = time.perf_counter() - t0
    value = system.n_springs * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload],
                       "impl": "FP64 CPU oracle: spring pass then mass pass, input order, one thread",
                       "accumulate": "serial spring loop in input order", "order": "input order (no reordering)",
                       "parallelism": "serial, rank 0 only", "l2": "not applicable (host)",
                       "sample": f"each timed step is one oracle step of the {system.n_masses}-mass "
                                 f"({system.n_springs}-spring) sub-lattice of the same recipe"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "nproc": host_cpu()[0], "cpu_model": host_cpu()[1],
                             "sample": f"each step: one FP64 oracle time step of a {system.name} "
                                       f"sub-lattice ({system.n_masses} masses, {system.n_springs} springs) "
                                       f"of the benchmark recipe, one thread"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_for(args, system, resolved=None):
    cfg = {"workload": WORKLOADS[args.workload],
           "accumulate": args.accumulate,
           "order": "input order (no reordering)" if args.order == "input"
           else ("grid cubes of 8x8x4 cells, Morton" if resolved in (6, 8, 9, 10) else "morton"),
           "graph_chunk": 64 if args.graph_chunk == 0 else args.graph_chunk,
           "csr_kernel": CSR_KERNELS.get(resolved, f"variant {args.kernel_variant}"),
           "parallelism": f"replicas x{args.gpus}", "exec": args.exec,
           "l2_persist": not getattr(args, "no_l2_persist", False),
           "launch_overlap": not getattr(args, "no_launch_overlap", False),
           "timing": "CUDA events on the simulation's stream, which a spin kernel holds while the host "
                     "enqueues the timed steps (device time of the steps, not host enqueue latency)",
           "l2": "inputs larger than L2 (spring data > 126 MB), no flush" if args.workload in ("lattice1m", "mesh2m")
           else "working set fits in L2 / shared memory, no flush (small-system latency case, not the headline)"}
    if system is not None:
        cfg.update({"masses": system.n_masses, "springs": system.n_springs})
    return cfg


def batched_leg(stream_handle, device, n_robots=4096, steps=2000, plain_robots=32, plain_steps=200, tune=True,
                robot_max=12):
    """Batched actuated robots (a, b, c ~ U{3..12}, 30% of springs actuated,
    ground contact): one rollout of `steps` steps for all robots in the
    persistent cluster launches, against plain per-robot launches (one kernel
    launch per robot per step) timed on a subset and expressed per rollout."""
    import torch
    from paper_1911_10274_gb300 import inputs
    from paper_1911_10274_gb300 import titan as T
    robots = inputs.robot_batch(n_robots, seed=0, hi=robot_max)
    springs = sum(r.n_springs for r in robots)
    with T.Batch(robots, device=device, stream=stream_handle) as b:
        if tune:
            b.autotune(50)
        times = []
        for _ in range(3):
            b.reset()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            b.rollout(steps)
            b.sync()
            times.append(time.perf_counter() - t0)
        groups = b.groups()
    t = min(times)
    sims = [T.Sim(r, graph_chunk=-1, device=device) for r in robots[:plain_robots]]
    for sm in sims:
        sm.step(10)
    for sm in sims:
        sm.sync()
    t0 = time.perf_counter()
    for _ in range(plain_steps):
        for sm in sims:
            T.titan_step(sm.handle, 1)
    for sm in sims:
        sm.sync()
    per_robot_step = (time.perf_counter() - t0) / (plain_steps * len(sims))
    for sm in sims:
        sm.close()
    plain = 1.0 / (per_robot_step * steps)
    return {"workload": f"{n_robots} actuated lattice robots, a,b,c ~ U{{3..{robot_max}}}, {springs} springs, "
                        f"{steps}-step rollouts, ground contact, dt=1e-4",
            "rollouts_per_s": n_robots / t, "plain_rollouts_per_s": plain, "speedup": n_robots / t / plain,
            "spring_updates_per_s": springs * steps / t, "rollout_s": t,
            "plain": f"one launch per robot per step, {plain_robots} robots x {plain_steps} steps",
            "launch_groups": groups}


def adjoint_leg(device, n_robots=4096, steps=200, every=50):
    """Adjoint of a 200-step rollout of the batched robots (centroid
    x-displacement w.r.t. every spring's actuation amplitude and phase),
    checkpointing every 50 steps; the robots are one block-diagonal system."""
    import torch
    from paper_1911_10274_gb300 import inputs
    from paper_1911_10274_gb300 import titan as T
    robots = inputs.robot_batch(n_robots, seed=0)
    f = T.CentroidRollout(robots, steps, every=every, device=device)
    amp = torch.tensor(f.system.act_amp, dtype=torch.float32, device=f"cuda:{device}")
    ph = torch.tensor(f.system.act_phase, dtype=torch.float32, device=f"cuda:{device}")
    g = torch.ones(n_robots, device=f"cuda:{device}")
    f.gradients(amp, ph, g)                      # warm-up (allocations, layouts)
    times = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        f.gradients(amp, ph, g)
        times.append(time.perf_counter() - t0)
    t = min(times)
    return {"workload": f"{n_robots} robots ({f.system.n_springs} springs), {steps}-step rollout, "
                        f"checkpoint every {every}", "seconds": t,
            "gradient_entries": 2 * f.system.n_springs, "adjoint_steps_per_s": steps / t,
            "note": "forward with checkpoints + per-segment recompute + two reverse kernels per step"}


def mlp_leg(device, batch=4096, n_in=1024, hidden=512, reps=20, big=True):
    """The surrogate's tensor-core work: the largest forward GEMM
    (batch x in) . (hidden x in)^T alone, and a whole training step."""
    import torch
    from paper_1911_10274_gb300 import titan as T
    dev = f"cuda:{device}"
    A = torch.randn(batch, n_in, device=dev).bfloat16()
    B = torch.randn(hidden, n_in, device=dev).bfloat16()
    C = torch.empty(batch, hidden, device=dev)
    for _ in range(3):
        T.titan_gemm_bf16_tn(A, B, C)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        T.titan_gemm_bf16_tn(A, B, C)            # enqueued back to back
    torch.cuda.synchronize()
    gemm_s = (time.perf_counter() - t0) / reps
    T.titan_gemm_check()
    flops = 2.0 * batch * n_in * hidden
    # the same kernel on a square 8192^3 product: its throughput once launch cost is amortised
    L = 8192
    AL = torch.randn(L, L, device=dev).bfloat16()
    BL = torch.randn(L, L, device=dev).bfloat16()
    CL = torch.empty(L, L, device=dev)
    for _ in range(3):
        T.titan_gemm_bf16_tn(AL, BL, CL)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(5):
        T.titan_gemm_bf16_tn(AL, BL, CL)
    torch.cuda.synchronize()
    large_s = (time.perf_counter() - t0) / 5
    T.titan_gemm_check()
    large_tflops = 2.0 * L ** 3 / large_s / 1e12
    del AL, BL, CL
    net = T.MLP(n_in, hidden, seed=0, device=device)

    def train_time(bsz, n):
        x = torch.randn(bsz, n_in, device=dev).bfloat16()
        t = torch.randn(bsz, device=dev)
        for _ in range(3):
            net.train_step(x, t, 1e-3)
        net.sync()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n):
            net.train_step(x, t, 1e-3)          # enqueued back to back (one captured graph each)
        net.sync()
        return (time.perf_counter() - t0) / n

    # forward: 3 products; backward: 3 weight-gradient products and the input
    # gradients of the two hidden layers (none for the network's input)
    def flops_of(bsz):
        return 2.0 * bsz * (3 * (n_in * hidden + 2 * hidden * hidden) - n_in * hidden)

    step_s = train_time(batch, reps)
    step_flops = flops_of(batch)
    big_batch = 8 * batch
    big_s = train_time(big_batch, reps) if big else None
    peak = bf16_peak()
    return {"gemm": f"{batch}x{hidden}x{n_in} BF16, FP32 accumulate (tcgen05)",
            "gemm_tflops": flops / gemm_s / 1e12, "gemm_s": gemm_s,
            "train_step_s": step_s, "train_samples_per_s": batch / step_s,
            "train_tflops": step_flops / step_s / 1e12,
            f"train_tflops_batch{big_batch}": flops_of(big_batch) / big_s / 1e12 if big else None,
            "gemm_8192_tflops": large_tflops, "gemm_8192_frac": large_tflops / peak[0],
            "roofline": {"bound": "tensor", "achieved": large_tflops, "peak": peak[0], "unit": "TFLOP/s",
                         "frac": large_tflops / peak[0], "peak_source": peak[1],
                         "kernel": "k_gemm_tn", "shape": f"{L}x{L}x{L}",
                         "note": "the kernel on a square product, 5 calls enqueued back to back and timed "
                                 "to the end of the last; at the MLP's own shapes (gemm_tflops) one call is a "
                                 "256-CTA launch (128 x 64 tiles, two per SM) of 4.3 GFLOP"}}


def bf16_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return float(json.load(open(p))["bf16_tflops"]), "measured cuBLAS BF16 burst"
    return 1900.0, "fallback"


def run_ours(args):
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1911_10274_gb300 import titan as T

    system = make_workload(args.workload)
    acc = T.ACCUM_CSR if args.accumulate == "csr" else T.ACCUM_ATOMIC
    stream = torch.cuda.Stream()            # a real stream: the legacy default stream is handle 0
    torch.cuda.set_stream(stream)
    exec_mode = {"auto": T.EXEC_AUTO, "launch": T.EXEC_LAUNCH, "persistent": T.EXEC_PERSISTENT}[args.exec]
    order = T.ORDER_MORTON if args.order == "morton" else T.ORDER_INPUT
    sim = T.Sim(system, accumulate=acc, stream=stream.cuda_stream, device=local,
                kernel_variant=args.kernel_variant, exec_mode=exec_mode, order=order,
                l2_persist=not args.no_l2_persist, launch_overlap=not args.no_launch_overlap,
                graph_chunk=args.graph_chunk)
    launches_per_step = 1 if acc == T.ACCUM_CSR else 2
    resolved = sim.csr_kernel
    persistent = sim.exec_mode == T.EXEC_PERSISTENT

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    with ClockSampler(local) as clocks:
        sim.step(args.warmup)
        # one untimed call with the timed step count: titan_step captures a
        # graph for a count of its own on first use, outside the timed region
        sim.step(args.steps)
        barrier()
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        # the stream is held by a spin kernel while the host enqueues the
        # start event and the K steps, so the events time the steps on the
        # device, not the host's enqueue latency (NVBench's blocking-kernel method)
        torch.cuda._sleep(QUEUE_FILL_CYCLES)
        start.record(stream)
        sim.step(args.steps)
        end.record(stream)
        barrier()
        ms = start.elapsed_time(end)
        # end-to-end through the C ABI with host buffers: upload state, K steps, read back
        pos0 = np.ascontiguousarray(system.pos)
        vel0 = np.ascontiguousarray(system.vel)
        # one untimed pass of the same calls first: the library allocates its
        # pinned staging and snapshot buffers on their first use
        sim.set_state(pos0, vel0)
        sim.step(args.steps)
        sim.snapshot(copy=False)
        # three timed passes, the median kept (host-side timings vary from pass to pass)
        passes = []
        for _ in range(E2E_PASSES):
            barrier()
            t0 = time.perf_counter()
            sim.set_state(pos0, vel0)
            sim.step(args.steps)
            p, v, _ = sim.snapshot(copy=False)       # the result in pinned host memory, read in place
            passes.append(time.perf_counter() - t0)
        e2e_s = sorted(passes)[len(passes) // 2]
        barrier()
    t_max, e2e_s = max_over_ranks([ms / 1e3, e2e_s], world, device="cuda")
    value = whole_job_rate(world, system.n_springs * args.steps, t_max)
    e2e_value = whole_job_rate(world, system.n_springs * args.steps, e2e_s)
    step_s = t_max / args.steps
    alg = algorithmic_bytes(system.n_masses, system.n_springs)
    peak, peak_kind = measured_peaks()
    achieved = alg / step_s / 1e9
    h = kernel_source_hash()
    kernel_name = "k_step_persist" if persistent else CSR_KERNEL_NAMES[resolved]
    traffic = NCU_TRAFFIC.get((args.workload, args.accumulate, kernel_name, h))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * step_s, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config_for(args, system, resolved),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": kernel_name,
                     "algorithmic_bytes_per_launch": alg,
                     "peak_source": f"{peak_kind} HBM copy bandwidth"},
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": 32 * system.n_masses / args.steps,
                "d2h_bytes_per_step": 24 * system.n_masses / args.steps,
                "note": "titan_set_state from host FP64 arrays, K steps, titan_snapshot into pinned host "
                        "memory (read in place, no further host copy); median of 3 passes after one "
                        "untimed pass"},
        "gpu_launches": -(-args.steps // 65536) if persistent else launches_per_step * args.steps,
        "clocks": clocks.summary(),
    }
    sim.close()
    if not args.no_batched:
        line["batched"] = batched_leg(stream.cuda_stream, local)
        line["adjoint"] = adjoint_leg(local)
        line["surrogate_mlp"] = mlp_leg(local)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_leg(system)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_leg(args):
    """One leg alone, for profiling: prints its JSON object."""
    import torch
    _, _, local = dist_env()
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    if args.leg == "batched":
        out = batched_leg(stream.cuda_stream, local, n_robots=args.robots, steps=args.rollout_steps,
                          plain_robots=min(32, args.robots), plain_steps=20, tune=not args.untuned,
                          robot_max=args.robot_max)
    elif args.leg == "adjoint":
        out = adjoint_leg(local, n_robots=args.robots, steps=args.rollout_steps)
    elif args.leg == "mlp":
        out = mlp_leg(local, reps=args.mlp_reps, big=not args.mlp_no_big)
    else:
        raise SystemExit(f"unknown leg {args.leg}")
    print(json.dumps({"leg": args.leg, **out}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=128)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--accumulate", choices=["csr", "atomic"], default="csr")
    ap.add_argument("--workload", default="lattice1m")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched-robots, adjoint and surrogate legs")
    ap.add_argument("--leg", choices=["batched", "adjoint", "mlp"], default=None,
                    help="run one secondary leg alone (for profiling) and print its JSON")
    ap.add_argument("--robots", type=int, default=4096, help="robots of the --leg batched/adjoint run")
    ap.add_argument("--rollout-steps", type=int, default=2000, help="rollout steps of the --leg run")
    ap.add_argument("--untuned", action="store_true", help="--leg batched: keep the default launch shapes")
    ap.add_argument("--robot-max", type=int, default=12, help="--leg batched: largest robot edge (masses)")
    ap.add_argument("--mlp-reps", type=int, default=20, help="--leg mlp: timed training steps per batch size")
    ap.add_argument("--mlp-no-big", action="store_true", help="--leg mlp: skip the 8x batch")
    ap.add_argument("--no-l2-persist", action="store_true",
                    help="do not keep the state buffers resident in L2 (access-policy window)")
    ap.add_argument("--order", choices=["morton", "input"], default="morton",
                    help="device order of the masses: spatial (grid cubes or Morton) or the caller's order")
    ap.add_argument("--exec", choices=["auto", "launch", "persistent"], default="auto",
                    help="step loop: persistent cluster kernel (small systems), per-step launches, or auto")
    ap.add_argument("--kernel-variant", type=int, default=0, help="CSR kernel: 0 auto, 1 direct loads, 2 TMA-staged, 3 bulk L2 prefetch, 4 halo, 5 halo+TMA, 6 grid box, 7 grid box+TMA, 8 cube")
    ap.add_argument("--graph-chunk", type=int, default=0,
                    help="steps per captured CUDA graph (0: the library default; < 0: direct launches)")
    ap.add_argument("--no-launch-overlap", action="store_true",
                    help="launch the step kernels in plain stream order (no programmatic dependent launch)")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.leg:
        run_leg(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

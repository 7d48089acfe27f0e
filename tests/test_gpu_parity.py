"""GPU (FP32, through the C ABI) vs the FP64 oracle, element by element.

Tolerance: the maximum position error must stay within 1e-4 of the lattice
spacing (1e-5 m for the 0.1 m lattices) after 1000 steps without contact and
after 100 steps with contact.  Velocities are checked at a looser bound derived
from the same position bound (velocity error ~ position error / (few dt)).
The deterministic (CSR) mode must be bit-identical from run to run.
"""
import numpy as np
import pytest

import oracle
from paper_1911_10274_gb300 import inputs
from paper_1911_10274_gb300 import titan as T

pytestmark = pytest.mark.gpu

POS_TOL_FRAC = 1e-4      # of the lattice spacing


def gpu_run(sys, steps, **kw):
    with T.Sim(sys, **kw) as sim:
        sim.step(steps)
        pos, vel, t = sim.snapshot()
    return pos.astype(np.float64), vel.astype(np.float64), t


def check(sys, steps, step0=0, spacing=None, **kw):
    spacing = sys.spacing if spacing is None else spacing
    xo, vo = oracle.run(sys, steps, step0=step0)
    xg, vg, t = gpu_run(sys, steps, **kw)
    err = np.abs(xg - xo).max()
    assert err <= POS_TOL_FRAC * spacing, f"max position error {err:.3e} > {POS_TOL_FRAC * spacing:.1e}"
    verr = np.abs(vg - vo).max()
    assert verr <= 1e3 * POS_TOL_FRAC * spacing, f"max velocity error {verr:.3e}"
    assert t == pytest.approx(steps * sys.dt, rel=1e-12)
    return err


LAUNCH = dict(exec_mode=T.EXEC_LAUNCH)      # one kernel per step: the variant choice applies
MODES = [dict(accumulate=T.ACCUM_CSR), dict(accumulate=T.ACCUM_ATOMIC),
         dict(accumulate=T.ACCUM_CSR, kernel_variant=1, **LAUNCH),
         dict(accumulate=T.ACCUM_CSR, kernel_variant=2, **LAUNCH),
         dict(accumulate=T.ACCUM_CSR, kernel_variant=3, **LAUNCH),
         dict(accumulate=T.ACCUM_CSR, kernel_variant=4, **LAUNCH),
         dict(accumulate=T.ACCUM_CSR, kernel_variant=5, **LAUNCH),
         dict(accumulate=T.ACCUM_CSR, kernel_variant=6, **LAUNCH),
         dict(accumulate=T.ACCUM_CSR, kernel_variant=7, **LAUNCH),
         dict(accumulate=T.ACCUM_CSR, kernel_variant=8, **LAUNCH),
         dict(accumulate=T.ACCUM_CSR, exec_mode=T.EXEC_PERSISTENT),
         dict(accumulate=T.ACCUM_CSR, order=T.ORDER_INPUT),
         dict(accumulate=T.ACCUM_CSR, graph_chunk=-1, **LAUNCH)]
MODE_IDS = ["csr", "atomic", "csr-direct-loads", "csr-tma-staged", "csr-bulk-prefetch", "csr-halo",
            "csr-halo-tma", "csr-grid-box", "csr-grid-box-tma", "csr-cube", "csr-persistent", "csr-input-order",
            "csr-no-graph"]


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
def test_cube_free_fall_1000_steps(mode):
    """Bouncing-cube workload, first 1000 steps (pure fall, no contact yet)."""
    check(inputs.cube_drop(), 1000, **mode)


def _contact_start():
    sys = inputs.cube_drop()
    x, v = oracle.run(sys, 3150)
    s2 = sys.copy()
    s2.pos, s2.vel = x, v
    return s2


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
def test_cube_contact_100_steps(mode):
    """From the oracle's state at step 3150 (just before the cube lands), 100
    steps through the first ground contact."""
    sys = _contact_start()
    xo, _ = oracle.run(sys, 100)
    assert xo[:, 2].min() < 0, "the window must contain ground contact"
    check(sys, 100, **mode)


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
def test_cube_penetrating_and_sliding_100_steps(mode):
    """Cube placed 1 mm into the ground, sliding at 0.1 m/s: penalty contact
    and capped Coulomb friction on every bottom mass from the first step."""
    sys = inputs.cube_drop(drop_height=-1e-3)
    sys.vel[:, 0] = 0.1
    sys.vel[:, 1] = -0.05
    check(sys, 100, **mode)


@pytest.mark.parametrize("mode", MODES[:7], ids=MODE_IDS[:7])
def test_cube_with_perturbed_rest_lengths_1000_steps(mode):
    """Same topology with rest lengths x U(0.95, 1.05) and lognormal k, so the
    internal spring forces are large from the first step."""
    sys = inputs.cube_drop(drop_height=2.0)
    rng = np.random.default_rng(7)
    sys.rest = sys.rest * rng.uniform(0.95, 1.05, sys.n_springs)
    sys.k = 1e4 * np.exp(0.5 * rng.standard_normal(sys.n_springs))
    check(sys, 1000, **mode)


def _zero_rest_grid():
    """The 10^3 cube (a grid: every kernel variant applies) with twelve springs
    of rest length 0 - legal input: such a spring pulls its ends together with
    force k l - softened to k = 300 so the lattice stays well conditioned."""
    sys = inputs.cube_drop(drop_height=0.3)
    rng = np.random.default_rng(21)
    idx = rng.choice(sys.n_springs, 12, replace=False)
    sys.rest[idx] = 0.0
    sys.k[idx] = 300.0
    sys.vel[:, 0] = 0.1
    return sys, idx


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
def test_grid_lattice_with_zero_rest_length_springs(mode):
    """Every kernel applies zero-rest-length springs (the grid kernels mark
    their padding by a negative rest length, never by a physical value);
    1000 steps of free fall, no contact."""
    sys, idx = _zero_rest_grid()
    without = sys.copy()
    without.k[idx] = 0.0
    xo, _ = oracle.run(sys, 1000)
    xw, _ = oracle.run(without, 1000)
    # the test is sensitive: dropping those springs moves masses far beyond the tolerance
    assert np.abs(xo - xw).max() > 100 * POS_TOL_FRAC * sys.spacing
    check(sys, 1000, **mode)


def test_zero_rest_length_springs_bit_identical_across_csr_kernels():
    sys, _ = _zero_rest_grid()
    a = gpu_run(sys, 500, exec_mode=T.EXEC_PERSISTENT)
    for var in range(1, 9):
        b = gpu_run(sys, 500, kernel_variant=var, **LAUNCH)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]), var


def _coincident_pair():
    """A 4^3 lattice plus one extra mass placed exactly on mass 0, joined to it
    by a spring whose rest length is NULL (the initial distance: 0) and to
    mass 1 by an ordinary one.  The pair starts with different velocities, so
    the zero-rest-length spring first has no axis (no force) and then pulls
    with k l as the masses separate."""
    base = inputs.cube_drop(n=4, drop_height=0.3)
    pos = np.concatenate([base.pos, base.pos[:1]])
    vel = np.zeros_like(pos)
    vel[-1] = (0.3, -0.2, 0.1)
    n = len(pos)
    ends = np.concatenate([base.ends, np.array([[0, n - 1], [n - 1, 1]], np.uint32)]).astype(np.uint32)
    k = np.concatenate([base.k, [2000.0, 1000.0]])
    rest = np.linalg.norm(pos[ends[:, 1]] - pos[ends[:, 0]], axis=1)
    assert rest[-2] == 0.0
    sys = inputs.System(pos=pos, vel=vel, mass=np.full(n, 0.1), fixed=np.zeros(n, np.uint8), ends=ends,
                        k=k, rest=rest, damping=np.full(len(ends), 1.0), dt=1e-4, ground=True, spacing=0.1)
    return sys


@pytest.mark.parametrize("mode", [m for m in MODES if m.get("kernel_variant") not in (6, 7, 8)],
                         ids=[i for m, i in zip(MODES, MODE_IDS) if m.get("kernel_variant") not in (6, 7, 8)])
def test_coincident_masses_joined_with_null_rest_length(mode):
    """Coincident masses are off-grid (one mass per cell), so the grid
    kernels do not apply; every other kernel is compared with the oracle,
    which is given the rest lengths the library derives from NULL."""
    sys = _coincident_pair()
    null_rest = sys.copy()
    null_rest.rest = None
    xo, vo = oracle.run(sys, 1000)
    assert np.linalg.norm(xo[-1] - xo[0]) > 1e-3          # they separated: the spring is stretched
    xg, vg, _ = gpu_run(null_rest, 1000, **mode)
    assert np.all(np.isfinite(xg))
    assert np.abs(xg - xo).max() <= POS_TOL_FRAC * sys.spacing
    assert np.abs(vg - vo).max() <= 1e3 * POS_TOL_FRAC * sys.spacing


def test_coincident_masses_are_refused_by_the_grid_kernels():
    sys = _coincident_pair()
    with pytest.raises(T.TitanError, match="grid"):
        T.Sim(sys, kernel_variant=6, **LAUNCH)


def test_per_spring_damping():
    sys = inputs.cube_drop(drop_height=2.0)
    rng = np.random.default_rng(3)
    sys.damping = rng.uniform(0.0, 3.0, sys.n_springs)
    sys.rest = sys.rest * rng.uniform(0.97, 1.03, sys.n_springs)
    check(sys, 1000)
    check(sys, 1000, accumulate=T.ACCUM_ATOMIC)


@pytest.mark.parametrize("accumulate", [T.ACCUM_CSR, T.ACCUM_ATOMIC], ids=["csr", "atomic"])
def test_large_lattice_scaled_down(accumulate):
    """The 1M-mass workload's recipe at 20^3: fixed bottom layer, perturbed
    rest lengths, lognormal k, no ground, dt = 5e-5, 1000 steps."""
    sys = inputs.large_lattice(n=20, seed=0)
    check(sys, 1000, accumulate=accumulate)
    xg, vg, _ = gpu_run(sys, 1000, accumulate=accumulate)
    fx = sys.fixed.astype(bool)
    assert np.array_equal(xg[fx], sys.pos[fx].astype(np.float32).astype(np.float64))
    assert np.all(vg[fx] == 0.0)


@pytest.mark.parametrize("order", [T.ORDER_INPUT, T.ORDER_MORTON], ids=["random-order", "morton"])
@pytest.mark.parametrize("variant", [0, 4, 3], ids=["auto", "halo", "bulk-prefetch"])
def test_random_mesh_scaled_down(order, variant):
    """Unstructured kNN mesh (random index order) at 5,000 points, ground on,
    dt = 2e-5, 500 steps; tolerance relative to the mean point spacing.  Not
    on a grid: Morton order and greedily coloured halo tables."""
    sys = inputs.random_mesh(n_points=5000, seed=1, lift=0.0)
    check(sys, 500, order=order, kernel_variant=variant, **(LAUNCH if variant else {}))


def test_lattice_with_holes_in_grid_tiles():
    """A 10 x 7 x 5 lattice does not fill whole 4 x 4 x 2 tiles: the grid-tile
    order leaves empty device slots that must stay inert."""
    pos = inputs.lattice_points(10, 7, 5, 0.1, (0.0, 0.0, 0.3))
    ends = inputs.lattice_springs(10, 7, 5)
    d = np.linalg.norm(pos[ends[:, 1]] - pos[ends[:, 0]], axis=1)
    rng = np.random.default_rng(9)
    sys = inputs.System(pos=pos, vel=rng.normal(0, 0.05, pos.shape), mass=np.full(len(pos), 0.1),
                        fixed=np.zeros(len(pos), np.uint8), ends=ends, k=np.full(len(ends), 1e4),
                        rest=d * rng.uniform(0.97, 1.03, len(d)), damping=np.full(len(ends), 1.0),
                        dt=1e-4, ground=True, spacing=0.1)
    for var in (0, 8, 7, 6, 5, 4, 3):
        check(sys, 1000, kernel_variant=var, **(LAUNCH if var else {}))


def test_actuated_robot_1000_steps():
    """One robot of the batched workload: a 6x4x3 lattice resting on the
    ground, 30% of springs actuated L0 (1 + A sin(2 pi 2 t + phi))."""
    sys = inputs.actuated_box(6, 4, 3, np.random.default_rng(11))
    assert (sys.act_amp > 0).any()
    check(sys, 1000)
    check(sys, 1000, accumulate=T.ACCUM_ATOMIC)


def test_actuation_set_mid_run_uses_absolute_time():
    """Actuation switched on after 300 steps uses t = step dt of the running
    simulation (not time since the call)."""
    sys = inputs.actuated_box(4, 4, 3, np.random.default_rng(5))
    plain = sys.copy()
    plain.act_amp = None
    x, v = oracle.run(plain, 300)
    mid = sys.copy()
    mid.pos, mid.vel = x, v
    xo, vo = oracle.run(mid, 200, step0=300)
    with T.Sim(plain) as sim:
        sim.step(300)
        T.titan_set_actuation(sim.handle, np.arange(sys.n_springs), sys.act_amp, sys.act_phase,
                              sys.act_freq)
        sim.step(200)
        xg, _, _ = sim.snapshot()
    assert np.abs(xg - xo).max() <= POS_TOL_FRAC * sys.spacing


def test_deterministic_mode_is_bit_exact_across_runs():
    sys = inputs.cube_drop(drop_height=0.05)
    sys.vel[:, 0] = 0.2
    a = gpu_run(sys, 2000)
    b = gpu_run(sys, 2000)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_resume_from_snapshot_is_bit_exact():
    """Resume on the same handle (set_state) and in a new handle (create from
    the snapshot, input order) both reproduce the uninterrupted run bit for bit."""
    sys = inputs.cube_drop(drop_height=0.05)
    sys.vel[:, 1] = 0.3
    full, _, _ = gpu_run(sys, 800, order=T.ORDER_INPUT)
    with T.Sim(sys, order=T.ORDER_INPUT) as sim:
        sim.step(400)
        p, v, _ = sim.snapshot()
        sim.set_state(p.astype(np.float64), v.astype(np.float64))
        sim.step(400)
        same, _, _ = sim.snapshot()
    s2 = sys.copy()
    s2.pos, s2.vel = p.astype(np.float64), v.astype(np.float64)
    fresh, _, _ = gpu_run(s2, 400, order=T.ORDER_INPUT)
    assert np.array_equal(same, full)
    assert np.array_equal(fresh, full)


def test_csr_kernel_variants_agree_bit_exact():
    """The CSR kernels (persistent cluster, grid box, halo, bulk-prefetched,
    direct, TMA-staged) sum the same entries in the same order: identical
    trajectories."""
    sys = inputs.cube_drop(drop_height=0.02)
    sys.vel[:, 0] = 0.3
    a = gpu_run(sys, 500, exec_mode=T.EXEC_PERSISTENT)
    for var in range(1, 9):
        b = gpu_run(sys, 500, kernel_variant=var, **LAUNCH)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]), var


def test_graph_ladder_and_launch_overlap_change_no_bit():
    """titan_step splits any step count into captured graphs of 64, 32, ...,
    2 steps plus at most one direct launch; step kernels launched as
    programmatic dependents (their CTAs start during the previous step's tail)
    or in plain stream order: every combination gives the same bits."""
    robot = inputs.actuated_box(9, 7, 5, np.random.default_rng(17))        # actuated: the step counter matters
    for sys in (inputs.large_lattice(n=20, seed=2), inputs.random_mesh(n_points=4000, seed=5, lift=0.0), robot):
        counts = [1, 2, 3, 5, 20, 63, 64, 65, 130]
        ref = None
        for kw in (dict(graph_chunk=-1, launch_overlap=False), dict(graph_chunk=-1), dict(launch_overlap=False), {}):
            with T.Sim(sys, **LAUNCH, **kw) as sim:
                for k in counts:
                    sim.step(k)
                x, v, t = sim.snapshot()
            assert t == pytest.approx(sum(counts) * sys.dt, rel=1e-12)
            if ref is None:
                ref = (x, v)
                if sys is robot:
                    xo, _ = oracle.run(robot, sum(counts))
                    assert np.abs(x - xo).max() <= POS_TOL_FRAC * robot.spacing
            else:
                assert np.array_equal(ref[0], x) and np.array_equal(ref[1], v), kw


def test_graph_replay_matches_direct_launches_bit_exact():
    sys = inputs.cube_drop(drop_height=0.02)
    a = gpu_run(sys, 300, graph_chunk=64)
    b = gpu_run(sys, 300, graph_chunk=-1)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


# --------------------------------------------------------------------------- edge cases

def test_single_mass_free_fall_and_empty_spring_list():
    sys = inputs.System(pos=np.array([[0.3, -0.2, 5.0]]), vel=np.array([[1.0, 0.0, 0.0]]),
                        mass=np.array([2.0]), fixed=np.zeros(1, np.uint8),
                        ends=np.zeros((0, 2), np.uint32), k=np.zeros(0), rest=np.zeros(0),
                        damping=np.zeros(0), dt=1e-3, ground=True, spacing=0.1)
    check(sys, 500)
    check(sys, 500, accumulate=T.ACCUM_ATOMIC)


def test_empty_system():
    sys = inputs.System(pos=np.zeros((0, 3)), vel=np.zeros((0, 3)), mass=np.zeros(0),
                        fixed=np.zeros(0, np.uint8), ends=np.zeros((0, 2), np.uint32),
                        k=np.zeros(0), rest=np.zeros(0), damping=np.zeros(0), dt=1e-3)
    for acc in (T.ACCUM_CSR, T.ACCUM_ATOMIC):
        pos, vel, t = gpu_run(sys, 10, accumulate=acc)
        assert pos.shape == (0, 3) and t == pytest.approx(0.01)


def test_ragged_sizes_and_zero_length_spring():
    """33 masses (one full slice plus one lane), uneven degrees, some fixed
    masses, and a spring whose two masses coincide and move together (zero
    length: no axis, no force, no NaN)."""
    rng = np.random.default_rng(4)
    n = 33
    pos = rng.uniform(0, 0.5, (n, 3))
    pos[5] = pos[4]
    vel = rng.normal(0, 0.1, (n, 3))
    vel[5] = vel[4]
    ends = [(4, 5)] + [(i, j) for i in range(n) for j in range(i + 1, n)
                       if i not in (4, 5) and j not in (4, 5) and rng.random() < 0.2]
    ends = np.array(ends, np.uint32)
    d = np.linalg.norm(pos[ends[:, 1]] - pos[ends[:, 0]], axis=1)
    fixed = (rng.random(n) < 0.1).astype(np.uint8)
    fixed[4] = fixed[5] = 0
    sys = inputs.System(pos=pos, vel=vel, mass=rng.uniform(0.05, 0.2, n), fixed=fixed, ends=ends,
                        k=rng.uniform(100, 1000, len(ends)), rest=d * rng.uniform(0.9, 1.1, len(ends)),
                        damping=np.full(len(ends), 0.1), dt=1e-4, gravity=(0, 0, -9.81), spacing=0.1)
    sys.rest[0] = 0.05
    sys.mass[5] = sys.mass[4]
    for acc in (T.ACCUM_CSR, T.ACCUM_ATOMIC):
        check(sys, 200, accumulate=acc)
        xg, vg, _ = gpu_run(sys, 200, accumulate=acc)
        assert np.all(np.isfinite(xg)) and np.array_equal(xg[4], xg[5])


def test_snapshot_tickets_and_double_buffer():
    sys = inputs.cube_drop(n=3)
    with T.Sim(sys) as sim:
        t1 = T.titan_snapshot_async(sim.handle)
        sim.step(10)
        t2 = T.titan_snapshot_async(sim.handle)
        sim.step(10)
        p2, _, tt2 = T.titan_snapshot_wait(sim.handle, t2, sim.n)
        p1, _, tt1 = T.titan_snapshot_wait(sim.handle, t1, sim.n)
        assert tt1 == 0.0 and tt2 == pytest.approx(10 * sys.dt)
        np.testing.assert_array_equal(p1, sys.pos.astype(np.float32))
        t3 = T.titan_snapshot_async(sim.handle)
        with pytest.raises(T.TitanError) as ei:
            T.titan_snapshot_wait(sim.handle, t1, sim.n)      # overwritten by t3
        assert ei.value.status == T.TITAN_E_INVALID
        p3, _, tt3 = T.titan_snapshot_wait(sim.handle, t3, sim.n)
        assert tt3 == pytest.approx(20 * sys.dt)
        xo, _ = oracle.run(sys, 20)
        assert np.abs(p3 - xo).max() <= POS_TOL_FRAC * sys.spacing


def test_read_state_into_torch_tensors():
    torch = pytest.importorskip("torch")
    sys = inputs.cube_drop(n=4)
    stream = torch.cuda.current_stream()
    with T.Sim(sys, stream=stream.cuda_stream) as sim:
        sim.step(50)
        pos = torch.empty((sim.n, 3), dtype=torch.float32, device="cuda")
        vel = torch.empty_like(pos)
        T.titan_read_state_dev(sim.handle, pos, vel, stream.cuda_stream)
        xo, vo = oracle.run(sys, 50)
        assert np.abs(pos.cpu().numpy() - xo).max() <= POS_TOL_FRAC * sys.spacing


def test_full_size_lattice_against_oracle_in_bench_configuration():
    """The 1M-mass, 12.7M-spring lattice in the benchmark's configuration
    (CSR, Morton order, 64-step graphs): 64 steps compared with the oracle on
    every mass, and the fixed bottom layer exactly still."""
    sys = inputs.large_lattice(n=100, seed=0)
    xo, vo = oracle.run(sys, 64)
    for mode in (dict(accumulate=T.ACCUM_CSR), dict(accumulate=T.ACCUM_CSR, kernel_variant=1, **LAUNCH),
                 dict(accumulate=T.ACCUM_CSR, kernel_variant=2, **LAUNCH),
                 dict(accumulate=T.ACCUM_CSR, kernel_variant=3, **LAUNCH),
                 dict(accumulate=T.ACCUM_CSR, kernel_variant=4, **LAUNCH),
                 dict(accumulate=T.ACCUM_CSR, kernel_variant=6, **LAUNCH),
                 dict(accumulate=T.ACCUM_CSR, kernel_variant=7, **LAUNCH),
                 dict(accumulate=T.ACCUM_CSR, kernel_variant=8, **LAUNCH),
                 dict(accumulate=T.ACCUM_ATOMIC)):
        xg, vg, _ = gpu_run(sys, 64, **mode)
        err = np.abs(xg - xo).max()
        assert err <= POS_TOL_FRAC * sys.spacing, err
        fx = sys.fixed.astype(bool)
        assert np.array_equal(xg[fx], sys.pos[fx].astype(np.float32).astype(np.float64))


def test_auto_kernel_choice():
    """Auto picks the persistent cluster kernel for systems that fit one
    cluster, else launches; among launch kernels the grid-box kernel for
    masses on a grid, the coloured halo kernel for an unstructured mesh; the
    cube kernel is taken when asked for on a 26-neighbour lattice; the box
    kernel refuses a mesh, the persistent mode a system too large."""
    with T.Sim(inputs.cube_drop(n=6)) as sim:
        assert sim.csr_kernel == 6 and sim.exec_mode == T.EXEC_PERSISTENT
    with T.Sim(inputs.cube_drop(n=6), exec_mode=T.EXEC_LAUNCH) as sim:
        assert sim.exec_mode == T.EXEC_LAUNCH
    big = inputs.large_lattice(n=20, seed=0)
    with T.Sim(big) as sim:
        assert sim.csr_kernel == 6 and sim.exec_mode == T.EXEC_LAUNCH
    with T.Sim(big, kernel_variant=8, exec_mode=T.EXEC_LAUNCH) as sim:
        assert sim.csr_kernel == 8
    with pytest.raises(T.TitanError, match="PERSISTENT"):
        T.Sim(big, exec_mode=T.EXEC_PERSISTENT)
    mesh = inputs.random_mesh(n_points=3000, seed=2, lift=0.0)
    with T.Sim(mesh, exec_mode=T.EXEC_LAUNCH) as sim:
        assert sim.csr_kernel == 4
    with T.Sim(mesh, accumulate=T.ACCUM_ATOMIC) as sim:
        assert sim.csr_kernel == 0
    with pytest.raises(T.TitanError, match="grid"):
        T.Sim(mesh, kernel_variant=6)


def test_grid_with_second_neighbour_springs_and_duplicates():
    """Springs two cells apart (same direction class as the nearest
    neighbour, a different cell offset) and a duplicated spring: the box
    kernel's offset-aligned columns hold them apart; all kernels agree with
    the oracle and with each other bit for bit."""
    n = 6
    pos = inputs.lattice_points(n, n, n, 0.1, (0.0, 0.0, 0.2))
    ends = inputs.lattice_springs(n, n, n)
    idx = np.arange(n ** 3).reshape(n, n, n)          # [z][y][x], as lattice_points numbers the sites
    far = np.stack([idx[:-2].ravel(), idx[2:].ravel()], 1)
    ends = np.concatenate([ends, far, ends[:7]]).astype(np.uint32)
    d = np.linalg.norm(pos[ends[:, 1]] - pos[ends[:, 0]], axis=1)
    rng = np.random.default_rng(4)
    sys = inputs.System(pos=pos, vel=rng.normal(0, 0.05, pos.shape), mass=np.full(len(pos), 0.1),
                        fixed=np.zeros(len(pos), np.uint8), ends=ends, k=rng.uniform(5e3, 2e4, len(ends)),
                        rest=d * rng.uniform(0.97, 1.03, len(d)), damping=np.full(len(ends), 1.0),
                        dt=1e-4, ground=True, spacing=0.1)
    with T.Sim(sys) as sim:
        assert sim.csr_kernel == 6                # second neighbours: no cube layout
    with pytest.raises(T.TitanError, match="cube"):
        T.Sim(sys, kernel_variant=8)
    runs = [gpu_run(sys, 400, kernel_variant=v, **LAUNCH) for v in (6, 7, 4, 3)]
    runs.append(gpu_run(sys, 400, exec_mode=T.EXEC_PERSISTENT))
    for r in runs[1:]:
        assert np.array_equal(runs[0][0], r[0]) and np.array_equal(runs[0][1], r[1])
    check(sys, 400)


def test_l2_persistence_changes_no_bit():
    """The L2 access-policy window on the state buffers is a cache hint: with
    and without it the trajectories are identical (grid-box and halo kernels)."""
    lattice = inputs.large_lattice(n=20, seed=0)
    mesh = inputs.random_mesh(n_points=4000, seed=3, lift=0.0)
    for sys in (lattice, mesh):
        a = gpu_run(sys, 200, l2_persist=True, **LAUNCH)
        b = gpu_run(sys, 200, l2_persist=False, **LAUNCH)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_snapshot_views_equal_copies_and_outlive_the_next_snapshot():
    """snapshot(copy=False) returns read-only views of the pinned snapshot
    buffers: the same values as a copy, still intact after one more snapshot."""
    sys = inputs.cube_drop(drop_height=0.02)
    with T.Sim(sys, **LAUNCH) as sim:
        sim.step(10)
        a = sim.snapshot()
        v = sim.snapshot(copy=False)
        assert np.array_equal(a[0], v[0]) and np.array_equal(a[1], v[1]) and a[2] == v[2]
        assert not v[0].flags.writeable and not v[1].flags.writeable
        sim.step(10)
        b = sim.snapshot()
        assert not np.array_equal(b[0], a[0])
        assert np.array_equal(v[0], a[0]) and np.array_equal(v[1], a[1])

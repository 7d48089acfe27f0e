"""The GPU adjoint (titan_adjoint, FP32) against the FP64 oracle's adjoint and
FP64 central finite differences (h = 1e-6) of the oracle's rollout.

Tolerance: 1e-3 relative, the bar the benchmark target sets for the adjoint,
read two ways.  Normwise: max absolute error <= 1e-3 x the largest gradient
entry.  Entry by entry: |g - ref| <= 1e-3 |ref| for every entry at least 1 %
of the largest (smaller entries are held to the normwise bound, 1e-3 of the
largest: their relative error is not meaningful at FP32 once they are
several orders of magnitude below it)."""
import numpy as np
import pytest

import oracle
from paper_1911_10274_gb300 import inputs
from paper_1911_10274_gb300 import titan as T

pytestmark = pytest.mark.gpu
REL = 1e-3


def _robot(dims=(5, 3, 3), seed=4, ground=True, all_actuated=False):
    rng = np.random.default_rng(seed)
    sy = inputs.actuated_box(*dims, rng)
    if all_actuated:
        sy.act_amp = rng.uniform(0.02, 0.2, sy.n_springs)
        sy.act_phase = rng.uniform(0, 2 * np.pi, sy.n_springs)
    sy.ground = ground
    if not ground:
        sy.gravity = (0.0, 0.0, 0.0)
    return sy


def _gpu_adjoint(sy, steps, seed, every=50, **kw):
    import torch
    with T.Sim(sy, **kw) as sim:
        s = torch.as_tensor(seed, dtype=torch.float32, device="cuda")
        ga = torch.empty(sy.n_springs, dtype=torch.float32, device="cuda")
        gp = torch.empty_like(ga)
        T.titan_adjoint(sim.handle, steps, every, s, None, ga, gp)
        sim.sync()
        x, _, t = sim.snapshot()
    return ga.cpu().numpy().astype(np.float64), gp.cpu().numpy().astype(np.float64), x, t


def _close(g, ref):
    scale = np.abs(ref).max()
    assert scale > 0
    err = np.abs(g - ref).max()
    assert err <= REL * scale, f"max error {err:.3e} vs {REL} x {scale:.3e}"
    big = np.abs(ref) >= 1e-2 * scale
    rel = np.abs(g[big] - ref[big]) / np.abs(ref[big])
    worst = int(np.flatnonzero(big)[np.argmax(rel)])
    assert rel.max() <= REL, (f"entry {worst}: {g[worst]:.6e} vs {ref[worst]:.6e} "
                              f"(relative {rel.max():.2e}; {big.sum()} entries checked)")


@pytest.mark.parametrize("ground", [False, True], ids=["floating", "on-ground"])
def test_adjoint_matches_oracle_adjoint(ground):
    sy = _robot(ground=ground, all_actuated=not ground)
    steps = 200
    rng = np.random.default_rng(0)
    seed = rng.standard_normal((sy.n_masses, 3)) if not ground else oracle.centroid_x_seed(sy.n_masses)
    ga, gp, xg, t = _gpu_adjoint(sy, steps, seed)
    ra, rp, xo, _ = oracle.adjoint(sy, steps, seed)
    _close(ga, ra)
    _close(gp, rp)
    assert np.abs(xg - xo).max() <= 1e-4 * sy.spacing      # the rollout itself advanced the state
    assert t == pytest.approx(steps * sy.dt)


def test_adjoint_matches_central_differences_on_the_benchmark_objective():
    """Centroid x-displacement after 200 steps, checkpoint every 50, robot on
    the ground: the GPU gradient against FP64 central differences."""
    sy = _robot(dims=(6, 4, 3), seed=9)
    steps = 200
    seed = oracle.centroid_x_seed(sy.n_masses)
    ga, gp, _, _ = _gpu_adjoint(sy, steps, seed, every=50)
    ra, rp, _, _ = oracle.adjoint(sy, steps, seed)
    _close(ga, ra)
    _close(gp, rp)
    scale_a, scale_p = np.abs(ra).max(), np.abs(rp).max()
    rng = np.random.default_rng(2)
    for s in rng.choice(np.flatnonzero(sy.act_amp > 0), 24, replace=False):
        for which, g, scale in (("amp", ga, scale_a), ("phase", gp, scale_p)):
            def J(delta):
                alt = sy.copy()
                arr = (alt.act_amp if which == "amp" else alt.act_phase).copy()
                arr[s] += delta
                if which == "amp":
                    alt.act_amp = arr
                else:
                    alt.act_phase = arr
                x, _ = oracle.run(alt, steps)
                return float((seed * x).sum())
            fd = (J(1e-6) - J(-1e-6)) / 2e-6
            # relative to the entry itself, floored at 1 % of the largest entry
            assert abs(g[s] - fd) <= REL * max(abs(fd), 1e-2 * scale), (which, s, g[s], fd)


def test_checkpoint_interval_does_not_change_the_result():
    sy = _robot(dims=(4, 4, 3), seed=3)
    seed = oracle.centroid_x_seed(sy.n_masses)
    a = _gpu_adjoint(sy, 120, seed, every=50)
    for every in (7, 120, 1):
        b = _gpu_adjoint(sy, 120, seed, every=every)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_adjoint_runs_in_every_csr_kernel_configuration():
    sy = _robot(dims=(4, 3, 3), seed=6)
    seed = oracle.centroid_x_seed(sy.n_masses)
    ref = _gpu_adjoint(sy, 100, seed)
    for kw in (dict(kernel_variant=3), dict(kernel_variant=1), dict(order=T.ORDER_INPUT)):
        g = _gpu_adjoint(sy, 100, seed, **kw)
        _close(g[0], ref[0])
        _close(g[1], ref[1])


def test_torch_autograd_function_over_several_robots():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(12)
    robots = [inputs.actuated_box(a, b, c, rng) for a, b, c in [(3, 3, 3), (5, 4, 3), (4, 3, 5)]]
    steps = 200
    f = T.CentroidRollout(robots, steps, every=50)
    amp = torch.tensor(f.system.act_amp, dtype=torch.float32, device="cuda", requires_grad=True)
    ph = torch.tensor(f.system.act_phase, dtype=torch.float32, device="cuda", requires_grad=True)
    J = f(amp, ph)
    assert J.shape == (3,)
    w = torch.tensor([1.0, -2.0, 0.5], device="cuda")
    (J * w).sum().backward()
    for r, sy in enumerate(robots):
        xo, _ = oracle.run(sy, steps)
        assert float(J[r].detach()) == pytest.approx(xo[:, 0].mean() - sy.pos[:, 0].mean(), abs=1e-5)
        ra, rp, _, _ = oracle.adjoint(sy, steps, oracle.centroid_x_seed(sy.n_masses))
        s0, s1 = f.spring_off[r], f.spring_off[r + 1]
        _close(amp.grad[s0:s1].cpu().numpy() / float(w[r]), ra)
        _close(ph.grad[s0:s1].cpu().numpy() / float(w[r]), rp)


def test_group_centroids_and_seed_match_numpy():
    """titan_group_centroids (mean position per group of caller indices, minus
    an origin) against the snapshot averaged in numpy; titan_group_seed
    against w[g] / |g| written by hand; an empty group gives 0."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    robots = [inputs.actuated_box(a, b, c, rng) for a, b, c in [(3, 3, 3), (4, 3, 2), (2, 2, 5)]]
    sy, mo, _ = T.union_system(robots)
    first = np.array([mo[0], mo[1], mo[1], mo[2], mo[3]], np.int32)      # group 1 is empty
    with T.Sim(sy) as sim:
        sim.step(57)
        x, _, _ = sim.snapshot()
        f = torch.as_tensor(first, device="cuda")
        origin = torch.as_tensor(rng.normal(0, 0.1, (4, 3)).astype(np.float32), device="cuda")
        out = torch.empty((4, 3), device="cuda")
        T.titan_group_centroids(sim.handle, f, origin, out)
        w = torch.tensor([0.5, 3.0, -1.0, 2.0], device="cuda")
        seed = torch.full((sy.n_masses, 3), 7.0, device="cuda")
        T.titan_group_seed(sim.handle, f, w, 1, seed)
        sim.sync()
    o = origin.cpu().numpy().astype(np.float64)
    got = out.cpu().numpy()
    for g in range(4):
        i0, i1 = first[g], first[g + 1]
        want = x[i0:i1].astype(np.float64).mean(axis=0) - o[g] if i1 > i0 else np.zeros(3)
        np.testing.assert_allclose(got[g], want, rtol=0, atol=1e-6)
    sd = seed.cpu().numpy()
    assert not sd[:, [0, 2]].any()
    wn = w.cpu().numpy().astype(np.float64)
    for g in range(4):
        i0, i1 = first[g], first[g + 1]
        if i1 > i0:
            np.testing.assert_array_equal(sd[i0:i1, 1], np.float32(wn[g] / (i1 - i0)))

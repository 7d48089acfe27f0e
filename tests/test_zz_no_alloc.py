"""The allocation-free atomic step (titan_step_atomic_noalloc), checked
against the regular atomic path built by titan_create.

Some callers cannot use cudaMalloc: a control loop with a hard per-step
deadline (the allocator may synchronise the device), or a plug-in whose host
framework owns all device memory.  For them the library keeps the atomic
scatter's force accumulator in a fixed array of its own.  This file is named
so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_1911_10274_gb300 import inputs
from paper_1911_10274_gb300 import titan as T

POS_TOL_FRAC = 1e-4        # of the lattice spacing, as in the parity tests
MAX_MASSES = 1 << 18


def _system():
    sys = inputs.cube_drop(drop_height=-1e-3)       # contact and friction from the first step
    sys.vel[:, 0] = 0.1
    rng = np.random.default_rng(12)
    sys.rest = sys.rest * rng.uniform(0.97, 1.03, sys.n_springs)   # internal forces too
    return sys


def _params(sys):
    p = T.titan_default_params()
    p.dt = sys.dt
    for a in range(3):
        p.gravity[a] = sys.gravity[a]
    p.ground = 1 if sys.ground else 0
    p.ground_k = sys.ground_k
    p.mu = sys.mu
    return p


def test_noalloc_rejects_counts_beyond_its_fixed_array():
    lib = T.load()
    p = T.titan_default_params()
    st = lib.titan_step_atomic_noalloc(MAX_MASSES + 1, None, None, None, 0, None, None, None, 0.0,
                                       p, None, None, None)
    assert st == T.TITAN_E_INVALID
    assert "static scratch limit" in T.titan_last_error(None)


@pytest.mark.gpu
def test_noalloc_step_matches_regular_atomic_step_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    sys = _system()
    assert np.all(sys.damping == sys.damping[0])
    with T.Sim(sys, accumulate=T.ACCUM_ATOMIC, order=T.ORDER_INPUT) as sim:
        ref = []
        for _ in range(2):
            sim.step(1)
            x, v, _ = sim.snapshot()
            ref.append((x.astype(np.float64), v.astype(np.float64)))

    dev = torch.device("cuda")
    f32 = dict(dtype=torch.float32, device=dev)
    pos = torch.tensor(sys.pos, **f32)
    vel = torch.tensor(sys.vel, **f32)
    inv_mass = torch.tensor(np.where(sys.fixed > 0, 0.0, 1.0 / sys.mass), **f32)
    ends = torch.tensor(sys.ends.astype(np.int32), dtype=torch.int32, device=dev)
    k = torch.tensor(sys.k, **f32)
    rest = torch.tensor(sys.rest, **f32)
    params = _params(sys)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        pos_out, vel_out = torch.empty_like(pos), torch.empty_like(vel)
        T.titan_step_atomic_noalloc(sys.n_masses, pos, vel, inv_mass, sys.n_springs, ends, k, rest,
                                    float(sys.damping[0]), params, pos_out, vel_out, stream)
        torch.cuda.synchronize()
        xr, vr = ref[call]
        err = np.abs(pos_out.cpu().numpy().astype(np.float64) - xr).max()
        verr = np.abs(vel_out.cpu().numpy().astype(np.float64) - vr).max()
        assert err <= POS_TOL_FRAC * sys.spacing, (call, err)
        assert verr <= 1e3 * POS_TOL_FRAC * sys.spacing, (call, verr)
        assert np.abs(vel_out.cpu().numpy() - vel.cpu().numpy()).max() > 0   # it did step
        pos, vel = pos_out, vel_out


def _gpu_tensors(sys, torch):
    dev = torch.device("cuda", torch.cuda.current_device())
    f32 = dict(dtype=torch.float32, device=dev)
    return dict(pos=torch.tensor(sys.pos, **f32), vel=torch.tensor(sys.vel, **f32),
                inv_mass=torch.tensor(np.where(sys.fixed > 0, 0.0, 1.0 / sys.mass), **f32),
                ends=torch.tensor(sys.ends.astype(np.int32), dtype=torch.int32, device=dev),
                k=torch.tensor(sys.k, **f32), rest=torch.tensor(sys.rest, **f32))


def _one_regular_step(sys):
    with T.Sim(sys, accumulate=T.ACCUM_ATOMIC, order=T.ORDER_INPUT) as sim:
        sim.step(1)
        x, v, _ = sim.snapshot()
    return x.astype(np.float64), v.astype(np.float64)


@pytest.mark.gpu
def test_noalloc_skips_and_reports_springs_with_bad_end_indices():
    """Spring ends are device data the host cannot see: a spring with an end
    beyond n_masses (inside the fixed array's range, so a missing check would
    corrupt it silently) or with both ends on one mass is skipped - the other
    masses step exactly as if it were absent - and the next call reports it
    with TITAN_E_INVALID without stepping; the call after that steps again."""
    torch = pytest.importorskip("torch")
    sys = _system()
    bad = [17, 40]
    broken = sys.copy()
    broken.ends[bad[0], 1] = sys.n_masses + 1000          # in [n_masses, 262144)
    broken.ends[bad[1], 1] = broken.ends[bad[1], 0]       # i == j
    keep = np.setdiff1d(np.arange(sys.n_springs), bad)
    absent = sys.copy()
    absent.ends, absent.k, absent.rest, absent.damping = (sys.ends[keep], sys.k[keep], sys.rest[keep],
                                                          sys.damping[keep])
    x_absent, v_absent = _one_regular_step(absent)
    x_full, v_full = _one_regular_step(sys)

    g = _gpu_tensors(broken, torch)
    good_ends = torch.tensor(sys.ends.astype(np.int32), dtype=torch.int32, device=g["ends"].device)
    params = _params(sys)
    stream = torch.cuda.current_stream().cuda_stream
    c = float(sys.damping[0])
    tol = POS_TOL_FRAC * sys.spacing

    out = torch.empty_like(g["pos"]), torch.empty_like(g["vel"])
    T.titan_step_atomic_noalloc(sys.n_masses, g["pos"], g["vel"], g["inv_mass"], sys.n_springs, g["ends"],
                                g["k"], g["rest"], c, params, *out, stream)
    torch.cuda.synchronize()
    assert np.abs(out[0].cpu().numpy() - x_absent).max() <= tol
    assert np.abs(out[1].cpu().numpy() - v_absent).max() <= 1e3 * tol

    out2 = torch.full_like(g["pos"], 7.0), torch.full_like(g["vel"], 7.0)
    with pytest.raises(T.TitanError) as ei:
        T.titan_step_atomic_noalloc(sys.n_masses, g["pos"], g["vel"], g["inv_mass"], sys.n_springs, good_ends,
                                    g["k"], g["rest"], c, params, *out2, stream)
    assert ei.value.status == T.TITAN_E_INVALID and "skipped 2 spring" in str(ei.value)
    torch.cuda.synchronize()
    assert torch.all(out2[0] == 7.0) and torch.all(out2[1] == 7.0)     # it did not step

    T.titan_step_atomic_noalloc(sys.n_masses, g["pos"], g["vel"], g["inv_mass"], sys.n_springs, good_ends,
                                g["k"], g["rest"], c, params, *out2, stream)
    torch.cuda.synchronize()
    assert np.abs(out2[0].cpu().numpy() - x_full).max() <= tol
    assert np.abs(out2[1].cpu().numpy() - v_full).max() <= 1e3 * tol


def test_noalloc_binding_checks_every_tensor_before_the_call():
    """The binding refuses, before any launch, what the C call would read or
    write blindly: host arrays, tensors on another device, wrong dtypes,
    non-contiguous views, wrong sizes and outputs overlapping an input."""
    torch = pytest.importorskip("torch")
    cpu = torch.device("cpu")
    n, s = 5, 4

    def args(**over):
        a = dict(pos=torch.zeros(n, 3), vel=torch.zeros(n, 3), inv_mass=torch.ones(n),
                 ends=torch.zeros(s, 2, dtype=torch.int32), k=torch.ones(s), rest=torch.ones(s),
                 pos_out=torch.zeros(n, 3), vel_out=torch.zeros(n, 3))
        a.update(over)
        return a

    def call(a):
        T.check_noalloc_args(n, s, a["pos"], a["vel"], a["inv_mass"], a["ends"], a["k"], a["rest"],
                             a["pos_out"], a["vel_out"], device=cpu)

    call(args())                                                    # the valid set passes
    with pytest.raises(TypeError, match="torch tensor"):
        call(args(pos=np.zeros((n, 3), np.float32)))
    with pytest.raises(ValueError, match="is on"):
        call(args(k=torch.ones(s, device="meta")))
    with pytest.raises(TypeError, match="dtype"):
        call(args(vel=torch.zeros(n, 3, dtype=torch.float64)))
    with pytest.raises(TypeError, match="dtype"):
        call(args(ends=torch.zeros(s, 2, dtype=torch.int64)))
    with pytest.raises(ValueError, match="contiguous"):
        call(args(pos=torch.zeros(3, n).t()))
    with pytest.raises(ValueError, match="elements"):
        call(args(inv_mass=torch.ones(n - 1)))
    with pytest.raises(ValueError, match="elements"):
        call(args(rest=torch.ones(s + 1)))
    pos = torch.zeros(n, 3)
    with pytest.raises(ValueError, match="overlaps pos"):
        call(args(pos=pos, pos_out=pos))
    big = torch.zeros(2 * 3 * n)
    with pytest.raises(ValueError, match="overlaps"):
        call(args(pos=big[:3 * n].view(n, 3), vel_out=big[3 * n - 3:6 * n - 3].view(n, 3)))
    if not torch.cuda.is_available():
        # the public wrapper refuses host tensors before it reaches the library
        with pytest.raises((TypeError, ValueError, RuntimeError, AssertionError)):
            a = args()
            T.titan_step_atomic_noalloc(n, a["pos"], a["vel"], a["inv_mass"], s, a["ends"], a["k"], a["rest"],
                                        0.0, T.titan_default_params(), a["pos_out"], a["vel_out"], None)

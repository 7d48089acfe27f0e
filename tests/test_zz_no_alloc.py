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

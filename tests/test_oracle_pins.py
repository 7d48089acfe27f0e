"""Pins of the FP64 oracle against facts fixed by the paper and by mechanics.

Each test targets a part of the time step (Titan Sec. III-B, Eq. 1 and the
Sec. III-A constraints) and is chosen so that a plausible slip in that part
(a dropped term, a flipped sign, a swapped index, a transposed component, the
wrong integrator ordering) fails it.  None of them re-types the oracle's own
formula: they compare against closed-form solutions, conservation laws,
symmetries and hand-evaluated special cases.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1911_10274_gb300 import inputs


def _no_env(sys):
    sys.gravity = (0.0, 0.0, 0.0)
    sys.ground = False
    return sys


def _jittered_lattice(n=4, seed=1, jitter=0.01, vscale=0.3, damping=0.5):
    rng = np.random.default_rng(seed)
    pos = inputs.lattice_points(n, n, n, 0.1) + rng.uniform(-jitter, jitter, (n ** 3, 3))
    ends = inputs.lattice_springs(n, n, n)
    s = ends.shape[0]
    base = inputs.lattice_points(n, n, n, 0.1)
    d = base[ends[:, 1]] - base[ends[:, 0]]
    rest = np.linalg.norm(d, axis=1) * rng.uniform(0.95, 1.05, s)
    return inputs.System(
        pos=pos, vel=rng.normal(0, vscale, (n ** 3, 3)), mass=rng.uniform(0.05, 0.2, n ** 3),
        fixed=np.zeros(n ** 3, np.uint8), ends=ends, k=1e4 * np.exp(0.5 * rng.standard_normal(s)),
        rest=rest, damping=np.full(s, damping), dt=1e-4, gravity=(0.0, 0.0, 0.0), ground=False)


# ----------------------------------------------------------------- integrator + gravity

def test_free_fall_matches_velocity_first_euler_closed_form():
    """No springs: x_n = x0 + n v0 dt + g dt^2 n(n+1)/2 exactly for the
    velocity-first Euler step that Eq. 1's dx = xdot dt + xddot dt^2 describes.
    A position-first step gives n(n-1)/2 and is off by g dt^2 n."""
    rng = np.random.default_rng(0)
    n = 7
    sys = inputs.System(pos=rng.uniform(-1, 1, (n, 3)), vel=rng.uniform(-2, 2, (n, 3)),
                        mass=rng.uniform(0.1, 1, n), fixed=np.zeros(n, np.uint8),
                        ends=np.zeros((0, 2), np.uint32), k=np.zeros(0), rest=np.zeros(0),
                        damping=np.zeros(0), dt=1e-3, gravity=(0.3, -0.2, -9.81), ground=False)
    steps = 1000
    x, v = oracle.run(sys, steps)
    g = np.array(sys.gravity)
    x_ref = sys.pos + steps * sys.vel * sys.dt + g * sys.dt ** 2 * steps * (steps + 1) / 2
    v_ref = sys.vel + steps * g * sys.dt
    np.testing.assert_allclose(x, x_ref, rtol=0, atol=1e-11)
    np.testing.assert_allclose(v, v_ref, rtol=0, atol=1e-11)


# ----------------------------------------------------------------- spring law

def _extension_history(sys, steps):
    x, v = sys.pos.copy(), sys.vel.copy()
    ext = np.empty(steps + 1)
    ext[0] = np.linalg.norm(x[1] - x[0]) - sys.rest[0]
    for n in range(steps):
        x, v = oracle.run(sys, 1, step0=n, pos=x, vel=v)
        ext[n + 1] = np.linalg.norm(x[1] - x[0]) - sys.rest[0]
    return ext


def _upward_crossings(ext, dt):
    idx = np.flatnonzero((ext[:-1] < 0) & (ext[1:] >= 0))
    return (idx + ext[idx] / (ext[idx] - ext[idx + 1])) * dt


def test_single_spring_period():
    """Undamped two-mass spring: period 2 pi sqrt(m_red / k) (0.01405 s for
    m = 0.1, k = 1e4), measured from zero crossings to 0.1%.  A flipped force
    sign has no crossings; a dropped rest length shifts the equilibrium."""
    sys = inputs.two_masses(stretch=1e-3, k=1e4, m=0.1, c=0.0, dt=1e-5)
    T = 2 * math.pi * math.sqrt(0.05 / 1e4)
    ext = _extension_history(sys, int(10.5 * T / sys.dt))
    t_up = _upward_crossings(ext, sys.dt)
    assert len(t_up) >= 9
    period = np.mean(np.diff(t_up))
    assert abs(period - T) / T < 1e-3
    # equilibrium is the rest length: the oscillation is centred on zero extension
    assert abs(ext.mean()) < 2e-5


def test_axial_damping_decay_rate():
    """Two masses with an axial dashpot c: m_red e'' + c e' + k e = 0, so the
    envelope decays as exp(-c t / (2 m_red)).  Checks successive peaks to 1%."""
    c = 0.5
    sys = inputs.two_masses(stretch=1e-3, k=1e4, m=0.1, c=c, dt=1e-5)
    T = 2 * math.pi * math.sqrt(0.05 / 1e4)
    ext = _extension_history(sys, int(8.2 * T / sys.dt))
    peaks = [i for i in range(1, len(ext) - 1) if ext[i] > ext[i - 1] and ext[i] >= ext[i + 1]
             and ext[i] > 0]
    assert len(peaks) >= 6
    t = np.array(peaks) * sys.dt
    rate = -np.polyfit(t, np.log(ext[peaks]), 1)[0]
    assert abs(rate - c / (2 * 0.05)) / (c / 0.1) < 1e-2


# ----------------------------------------------------------------- conservation

def test_internal_forces_sum_to_zero():
    sys = _jittered_lattice()
    F = oracle.spring_forces(sys)
    assert np.abs(F).max() > 1.0
    np.testing.assert_allclose(F.sum(axis=0), 0.0, atol=1e-10 * np.abs(F).max() * len(F))


def test_linear_and_angular_momentum_conserved():
    """Gravity and ground off: pairwise forces along the spring axis conserve
    total momentum, and for central forces velocity-first Euler conserves
    L = sum(x x m v) exactly: L_{n+1} = L_n + dt sum(x_n x F_n) and every
    pair contributes (x_i - x_j) x f u = 0.  A dashpot acting along
    (v_j - v_i) instead of the axis, or a transposed component, breaks it."""
    sys = _jittered_lattice(damping=2.0)
    m = sys.mass[:, None]

    def momenta(x, v):
        return (m * v).sum(axis=0), np.cross(x, m * v).sum(axis=0)

    P0, L0 = momenta(sys.pos, sys.vel)
    x, v = oracle.run(sys, 500)
    P1, L1 = momenta(x, v)
    assert np.abs(v - sys.vel).max() > 0.1          # the springs did work
    np.testing.assert_allclose(P1, P0, atol=1e-12 * (1 + np.abs(P0).max()))
    scale = np.abs(np.cross(x, m * v)).sum()
    np.testing.assert_allclose(L1, L0, atol=1e-12 * scale)


def test_energy_drift_bounded_without_damping():
    """c = 0, no gravity or ground: symplectic Euler keeps the energy error
    bounded over 10^4 steps (it oscillates around a shadow energy, with no
    secular growth), and the oscillation is first order in dt: halving dt
    halves it.  A forward (non-symplectic) Euler step grows without bound."""
    def fluctuation(dt, t_end=1.0):
        sys = _jittered_lattice(n=5, damping=0.0, vscale=0.2, jitter=0.005)
        sys.mass[:] = 0.1
        sys.dt = dt

        def energy(x, v):
            d = x[sys.ends[:, 1]] - x[sys.ends[:, 0]]
            ext = np.linalg.norm(d, axis=1) - sys.rest
            return 0.5 * (sys.mass[:, None] * v * v).sum() + 0.5 * (sys.k * ext * ext).sum()

        x, v = sys.pos.copy(), sys.vel.copy()
        E = [energy(x, v)]
        chunk = int(round(0.01 / dt))
        for n in range(0, int(round(t_end / dt)), chunk):
            x, v = oracle.run(sys, chunk, step0=n, pos=x, vel=v)
            E.append(energy(x, v))
        E = np.array(E)
        q = len(E) // 4
        drift = abs(E[-q:].mean() - E[1:q + 1].mean()) / E[0]
        return np.abs(E - E[0]).max() / E[0], drift

    f1, d1 = fluctuation(1e-4)
    f2, d2 = fluctuation(5e-5)
    assert f1 < 0.03 and d1 < 1e-3 and d2 < 1e-3
    assert 1.5 < f1 / f2 < 2.5


# ----------------------------------------------------------------- symmetries

def test_rotation_equivariance():
    """Rotating the initial state rotates the trajectory (no gravity/ground)."""
    sys = _jittered_lattice()
    rng = np.random.default_rng(5)
    q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    x, v = oracle.run(sys, 200)
    xr, vr = oracle.run(sys, 200, pos=sys.pos @ q.T, vel=sys.vel @ q.T)
    np.testing.assert_allclose(xr, x @ q.T, atol=1e-10)
    np.testing.assert_allclose(vr, v @ q.T, atol=1e-8)


def test_spring_order_and_orientation_do_not_matter():
    """Permuting the spring list and swapping the two ends of half the springs
    changes results only by summation rounding."""
    sys = _jittered_lattice()
    rng = np.random.default_rng(2)
    perm = rng.permutation(sys.n_springs)
    alt = sys.copy()
    alt.ends = sys.ends[perm].copy()
    flip = rng.random(sys.n_springs) < 0.5
    alt.ends[flip] = alt.ends[flip][:, ::-1]
    alt.k, alt.rest, alt.damping = sys.k[perm], sys.rest[perm], sys.damping[perm]
    x, v = oracle.run(sys, 200)
    xa, va = oracle.run(alt, 200)
    np.testing.assert_allclose(xa, x, atol=1e-11)
    np.testing.assert_allclose(va, v, atol=1e-8)


def test_mass_relabelling_equivariance():
    sys = _jittered_lattice()
    rng = np.random.default_rng(3)
    perm = rng.permutation(sys.n_masses)      # new index -> old index
    inv = np.argsort(perm)
    alt = sys.copy()
    alt.pos, alt.vel, alt.mass = sys.pos[perm], sys.vel[perm], sys.mass[perm]
    alt.ends = inv[sys.ends.astype(np.int64)].astype(np.uint32)
    x, v = oracle.run(sys, 100)
    xa, va = oracle.run(alt, 100)
    np.testing.assert_allclose(xa, x[perm], atol=1e-12)


# ----------------------------------------------------------------- constraints and contact

def test_fixed_masses_never_move():
    sys = inputs.large_lattice(n=5, seed=0)
    sys.vel[:] = 0.3
    x, v = oracle.run(sys, 300)
    fx = sys.fixed.astype(bool)
    assert fx.sum() == 25
    assert np.array_equal(x[fx], sys.pos[fx])
    assert np.all(v[fx] == 0.0)
    assert np.abs(x[~fx] - sys.pos[~fx]).max() > 1e-3


def test_cube_rests_on_ground_with_normal_force_equal_to_weight():
    """A damped cube settled on the ground: the penalty forces sum to M g
    (the static equilibrium of the external forces), and the bottom layer's
    mean penetration is M g / (n_bottom k_g)."""
    sys = inputs.cube_drop(n=3, drop_height=0.002)
    sys.damping[:] = 20.0
    x, v = oracle.run(sys, 30000)
    M = sys.mass.sum()
    g = 9.81
    below = np.maximum(0.0, -x[:, 2])
    assert np.abs(v).max() < 1e-4
    assert abs(sys.ground_k * below.sum() - M * g) / (M * g) < 1e-3
    bottom = x[:9, 2]
    assert abs(-bottom.mean() - M * g / (9 * sys.ground_k)) / (M * g / (9 * sys.ground_k)) < 0.05


def test_coulomb_friction_decelerates_at_mu_g_then_stops():
    """One mass sliding on the ground at its equilibrium depth decelerates at
    mu g, stops at t = v0 / (mu g) after sliding v0^2 / (2 mu g), and does not
    reverse (friction is capped at m |v_t| / dt)."""
    m, kg, mu, g, v0, dt = 0.1, 1e5, 0.5, 9.81, 0.5, 1e-4
    sys = inputs.System(pos=np.array([[0.0, 0.0, -m * g / kg]]), vel=np.array([[v0, 0.0, 0.0]]),
                        mass=np.array([m]), fixed=np.zeros(1, np.uint8),
                        ends=np.zeros((0, 2), np.uint32), k=np.zeros(0), rest=np.zeros(0),
                        damping=np.zeros(0), dt=dt, ground=True, ground_k=kg, mu=mu)
    x, v = sys.pos.copy(), sys.vel.copy()
    vx = [v0]
    for n in range(1500):
        x, v = oracle.run(sys, 1, step0=n, pos=x, vel=v)
        vx.append(v[0, 0])
    vx = np.array(vx)
    t_stop = v0 / (mu * g)
    n_stop = int(np.argmax(vx == 0.0))
    assert n_stop > 0 and abs(n_stop * dt - t_stop) < 2 * dt
    np.testing.assert_allclose(np.diff(vx[:n_stop - 1]) / dt, -mu * g, rtol=1e-6)
    assert np.all(vx[n_stop:] == 0.0)
    assert abs(x[0, 0] - v0 ** 2 / (2 * mu * g)) < v0 * dt


def test_ground_off_means_no_contact():
    sys = inputs.cube_drop(n=2, drop_height=-0.5)
    sys.ground = False
    x, v = oracle.run(sys, 10)
    # pure free fall of a rigid cube at rest length
    np.testing.assert_allclose(v[:, 2], -9.81 * 10 * sys.dt, rtol=1e-9)


# ----------------------------------------------------------------- actuation

def test_actuated_spring_follows_driven_oscillator_steady_state():
    """One spring with L(t) = L0 (1 + A sin(2 pi f t + phi)) between two
    masses: the extension y = l - L0 obeys m_red y'' + c y' + k y =
    k L0 A sin(2 pi f t + phi), whose steady state is the textbook driven
    oscillator response.  Pins the 2 pi, the phase sign and the amplitude."""
    k, m, L0, A, f, phi, dt = 1e4, 0.1, 0.1, 0.1, 2.0, 0.7, 1e-5
    mr = m / 2
    c = 2 * math.sqrt(k * mr)                     # critical damping: transients die fast
    sys = inputs.two_masses(stretch=0.0, k=k, m=m, c=c, length=L0, dt=dt)
    sys.act_amp, sys.act_phase, sys.act_freq = np.array([A]), np.array([phi]), f
    W = 2 * math.pi * f
    H = 1.0 / math.sqrt((k - mr * W * W) ** 2 + (c * W) ** 2)
    delta = math.atan2(c * W, k - mr * W * W)
    x, v = sys.pos.copy(), sys.vel.copy()
    n0 = 20000                                  # 0.2 s: transients are gone
    x, v = oracle.run(sys, n0, pos=x, vel=v)
    err = 0.0
    for n in range(n0, n0 + 50000, 500):
        y = np.linalg.norm(x[1] - x[0]) - L0
        y_ref = H * k * L0 * A * math.sin(W * n * dt + phi - delta)
        err = max(err, abs(y - y_ref))
        x, v = oracle.run(sys, 500, step0=n, pos=x, vel=v)
    assert err < 2e-3 * (H * k * L0 * A)


def test_actuation_rest_length_hand_values():
    """Hand-evaluated special cases of both actuation forms.
    Sinusoid, A = 0.2, f = 1 Hz, phi = 0: at t = 0.25 s, L = 1.2 L0; at 0.5 s, L0.
    Worm (Sec. IV-B, Eqs. 3-4; t_p = 1 s, omega = 20, c = 0.2 as printed there):
    with t_o = 0.1, T = 0.3 gives tau = 0.2 and T = 0.05 wraps to tau = 0.95."""
    sys = inputs.two_masses()
    sys.act_amp, sys.act_phase, sys.act_freq = np.array([0.2]), np.array([0.0]), 1.0
    assert oracle.rest_length(sys, 0, 0.25) == pytest.approx(1.2 * 0.1, rel=1e-14)
    assert oracle.rest_length(sys, 0, 0.5) == pytest.approx(0.1, rel=1e-14)
    sys.act_phase = np.array([0.1])
    worm = (20.0, 1.0)
    assert oracle.rest_length(sys, 0, 0.3, act_mode=2, worm=worm) == pytest.approx(
        0.1 * (1 + 0.2 * math.sin(20 * 0.2)), rel=1e-12)
    assert oracle.rest_length(sys, 0, 0.05, act_mode=2, worm=worm) == pytest.approx(
        0.1 * (1 + 0.2 * math.sin(20 * 0.95)), rel=1e-12)
    # the force of a spring held at L0 at t = 0.25 s with A = 0.2 is -0.2 k L0
    sys.act_phase = np.array([0.0])
    sys.dt = 0.25
    F = oracle.spring_forces(sys, pos=np.array([[0.0, 0, 0], [0.1, 0, 0]]), step=1)
    assert F[0, 0] == pytest.approx(-0.2 * 1e4 * 0.1, rel=1e-12)
    assert F[1, 0] == pytest.approx(+0.2 * 1e4 * 0.1, rel=1e-12)


def test_zero_length_spring_applies_no_force():
    sys = inputs.two_masses()
    F = oracle.spring_forces(sys, pos=np.zeros((2, 3)))
    assert np.all(F == 0.0)

"""Seeded synthetic inputs for the spring-mass hot path.

This module builds input systems only: lattice and mesh geometry, spring lists,
stiffness and rest-length draws, robot morphologies.  It holds none of the time
step's arithmetic (no force, no integration), and it imports neither the CUDA
path nor the oracle; both of those consume what it returns.

Workload shapes follow the paper's experiments: n^3 cubic lattices with springs
to every 26-neighbourhood lattice neighbour (Sec. V-A; a 50^3 lattice has
exactly 1,558,396 such springs, the count the paper prints), rectangular
actuated lattices (Sec. V-B worms), plus the larger single-body, unstructured
mesh, robot-batch and voxel-morphology workloads of the benchmark suite.
All draws use numpy's PCG64 generator from an explicit seed.
"""
from __future__ import annotations

import dataclasses
from typing import Optional, Tuple

import numpy as np

# The 13 lattice offsets that point "forward" (first non-zero component > 0 in
# (dz, dy, dx) order).  Together with their negatives they are the 26
# neighbours of a cubic lattice site: 3 axis, 6 face-diagonal, 4 body-diagonal.
FORWARD_OFFSETS = np.array(
    [(dx, dy, dz)
     for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
     if (dz, dy, dx) > (0, 0, 0)],
    dtype=np.int64)
assert FORWARD_OFFSETS.shape == (13, 3)


@dataclasses.dataclass
class System:
    """A spring-mass system and its integration parameters (SI units, FP64).

    pos, vel: (n, 3); mass: (n,); fixed: (n,) uint8 (1 = fixed mass).
    ends: (s, 2) uint32 end-mass indices; k, rest, damping: (s,).
    act_amp/act_phase: (s,) or None (mode 1: L0 (1 + A sin(2 pi f t + phi))).
    """
    pos: np.ndarray
    vel: np.ndarray
    mass: np.ndarray
    fixed: np.ndarray
    ends: np.ndarray
    k: np.ndarray
    rest: np.ndarray
    damping: np.ndarray
    dt: float
    gravity: Tuple[float, float, float] = (0.0, 0.0, -9.81)
    ground: bool = False
    ground_k: float = 1e5
    mu: float = 0.5
    act_amp: Optional[np.ndarray] = None
    act_phase: Optional[np.ndarray] = None
    act_freq: float = 0.0
    spacing: float = 0.1
    name: str = ""

    @property
    def n_masses(self) -> int:
        return int(self.pos.shape[0])

    @property
    def n_springs(self) -> int:
        return int(self.ends.shape[0])

    def copy(self) -> "System":
        return dataclasses.replace(
            self, **{f.name: (getattr(self, f.name).copy()
                              if isinstance(getattr(self, f.name), np.ndarray) else getattr(self, f.name))
                     for f in dataclasses.fields(self)})


# --------------------------------------------------------------------------- lattices

def lattice_points(nx: int, ny: int, nz: int, spacing: float, origin=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Sites of an nx x ny x nz cubic lattice, index = ix + nx (iy + ny iz)."""
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    p = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64) * spacing
    return p + np.asarray(origin, dtype=np.float64)


def lattice_springs(nx: int, ny: int, nz: int, occupied: Optional[np.ndarray] = None) -> np.ndarray:
    """All 26-neighbourhood pairs of an nx x ny x nz lattice, each pair once.

    ``occupied`` (optional, bool (nz, ny, nx)) drops pairs that touch an empty
    site; the returned indices still address the full lattice.  Pairs come out
    grouped by offset (in FORWARD_OFFSETS order), then by the first site's
    index, with the first site the one the offset points away from.
    """
    idx = np.arange(nx * ny * nz, dtype=np.int64).reshape(nz, ny, nx)
    occ = np.ones((nz, ny, nx), dtype=bool) if occupied is None else occupied
    out = []
    for dx, dy, dz in FORWARD_OFFSETS:
        xs0, xs1 = max(0, -dx), nx - max(0, dx)
        ys0, ys1 = max(0, -dy), ny - max(0, dy)
        zs0, zs1 = max(0, -dz), nz - max(0, dz)
        if xs1 <= xs0 or ys1 <= ys0 or zs1 <= zs0:
            continue
        a = idx[zs0:zs1, ys0:ys1, xs0:xs1]
        b = idx[zs0 + dz:zs1 + dz, ys0 + dy:ys1 + dy, xs0 + dx:xs1 + dx]
        keep = occ[zs0:zs1, ys0:ys1, xs0:xs1] & occ[zs0 + dz:zs1 + dz, ys0 + dy:ys1 + dy, xs0 + dx:xs1 + dx]
        out.append(np.stack([a[keep], b[keep]], axis=1))
    if not out:
        return np.zeros((0, 2), dtype=np.uint32)
    return np.concatenate(out).astype(np.uint32)


def lattice_spring_count(nx: int, ny: int, nz: int) -> int:
    """Closed-form count of 26-neighbourhood pairs: axis + face + body diagonals."""
    axis = (nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1)
    face = 2 * ((nx - 1) * (ny - 1) * nz + (nx - 1) * ny * (nz - 1) + nx * (ny - 1) * (nz - 1))
    body = 4 * (nx - 1) * (ny - 1) * (nz - 1)
    return axis + face + body


def _initial_lengths(pos: np.ndarray, ends: np.ndarray) -> np.ndarray:
    d = pos[ends[:, 1].astype(np.int64)] - pos[ends[:, 0].astype(np.int64)]
    return np.sqrt(np.einsum("ij,ij->i", d, d))


# --------------------------------------------------------------------------- workloads

def cube_drop(n: int = 10, spacing: float = 0.1, mass: float = 0.1, k: float = 1e4,
              damping: float = 1.0, drop_height: float = 0.5, dt: float = 1e-4,
              ground_k: float = 1e5, mu: float = 0.5) -> System:
    """Bouncing-cube workload (Sec. V-A): an n^3 lattice dropped onto the ground.

    10^3 sites, 10,476 springs, k = 1e4, c = 1, rest length = initial distance,
    lowest layer at z = drop_height, at rest, ground k_g = 1e5 and mu = 0.5.
    """
    pos = lattice_points(n, n, n, spacing, (0.0, 0.0, drop_height))
    ends = lattice_springs(n, n, n)
    s = ends.shape[0]
    return System(pos=pos, vel=np.zeros_like(pos), mass=np.full(n ** 3, mass),
                  fixed=np.zeros(n ** 3, np.uint8), ends=ends, k=np.full(s, k),
                  rest=_initial_lengths(pos, ends), damping=np.full(s, damping), dt=dt,
                  ground=True, ground_k=ground_k, mu=mu, spacing=spacing,
                  name=f"cube{n}_drop")


def large_lattice(n: int = 100, seed: int = 0, spacing: float = 0.1, mass: float = 0.1,
                  k_median: float = 1e4, k_sigma: float = 0.5, rest_jitter: float = 0.05,
                  damping: float = 1.0, dt: float = 5e-5) -> System:
    """Large single-body lattice: n^3 sites, rest lengths = distance x U(1-j, 1+j),
    k lognormal (median k_median, sigma k_sigma), bottom layer fixed, no ground.

    At n = 100: 1,000,000 masses and 12,731,796 springs.
    """
    rng = np.random.default_rng(seed)
    pos = lattice_points(n, n, n, spacing)
    ends = lattice_springs(n, n, n)
    s = ends.shape[0]
    rest = _initial_lengths(pos, ends) * rng.uniform(1.0 - rest_jitter, 1.0 + rest_jitter, s)
    kk = k_median * np.exp(k_sigma * rng.standard_normal(s))
    fixed = np.zeros(n ** 3, np.uint8)
    fixed[: n * n] = 1                      # iz == 0 layer
    return System(pos=pos, vel=np.zeros_like(pos), mass=np.full(n ** 3, mass), fixed=fixed,
                  ends=ends, k=kk, rest=rest, damping=np.full(s, damping), dt=dt, ground=False,
                  spacing=spacing, name=f"lattice{n}_fixed_base")


def knn_pairs(pos: np.ndarray, knn: int) -> np.ndarray:
    """Undirected, de-duplicated pairs {i, j} with j among the knn nearest of i."""
    from scipy.spatial import cKDTree
    tree = cKDTree(pos)
    _, nb = tree.query(pos, k=knn + 1)
    i = np.repeat(np.arange(pos.shape[0], dtype=np.int64), knn)
    j = nb[:, 1:].reshape(-1).astype(np.int64)
    lo, hi = np.minimum(i, j), np.maximum(i, j)
    key = np.unique(lo * pos.shape[0] + hi)
    return np.stack([key // pos.shape[0], key % pos.shape[0]], axis=1).astype(np.uint32)


def random_mesh(n_points: int = 2_000_000, knn: int = 8, seed: int = 0, k: float = 5e3,
                damping: float = 0.5, mass: float = 1e-3, dt: float = 2e-5,
                ground_k: float = 1e5, mu: float = 0.5, lift: float = 0.0) -> System:
    """Unstructured mesh: n points uniform in the unit cube (random index order),
    springs to each point's knn nearest neighbours, de-duplicated, rest length =
    initial distance, ground contact on."""
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0.0, 1.0, (n_points, 3))
    pos[:, 2] += lift
    ends = knn_pairs(pos, knn)
    order = rng.permutation(ends.shape[0])          # springs in random order as well
    ends = ends[order]
    s = ends.shape[0]
    mean_spacing = float(np.cbrt(1.0 / n_points))
    return System(pos=pos, vel=np.zeros_like(pos), mass=np.full(n_points, mass),
                  fixed=np.zeros(n_points, np.uint8), ends=ends, k=np.full(s, k),
                  rest=_initial_lengths(pos, ends), damping=np.full(s, damping), dt=dt,
                  ground=True, ground_k=ground_k, mu=mu, spacing=mean_spacing,
                  name=f"mesh{n_points}_knn{knn}")


def actuated_box(a: int, b: int, c: int, rng: np.random.Generator, spacing: float = 0.1,
                 mass: float = 0.1, k: float = 1e4, damping: float = 1.0, act_prob: float = 0.3,
                 amp_max: float = 0.2, origin=(0.0, 0.0, 0.0)) -> System:
    """One a x b x c lattice robot resting on the ground (lowest layer at z = 0),
    with a Bernoulli(act_prob) subset of springs actuated, A ~ U[0, amp_max],
    phi ~ U[0, 2 pi); non-actuated springs have A = 0."""
    pos = lattice_points(a, b, c, spacing, origin)
    ends = lattice_springs(a, b, c)
    s = ends.shape[0]
    act = rng.random(s) < act_prob
    amp = np.where(act, rng.uniform(0.0, amp_max, s), 0.0)
    phase = np.where(act, rng.uniform(0.0, 2.0 * np.pi, s), 0.0)
    return System(pos=pos, vel=np.zeros_like(pos), mass=np.full(pos.shape[0], mass),
                  fixed=np.zeros(pos.shape[0], np.uint8), ends=ends, k=np.full(s, k),
                  rest=_initial_lengths(pos, ends), damping=np.full(s, damping), dt=1e-4,
                  ground=True, ground_k=1e5, mu=0.5, act_amp=amp, act_phase=phase,
                  act_freq=2.0, spacing=spacing, name=f"box{a}x{b}x{c}")


def robot_batch(n_robots: int = 4096, seed: int = 0, lo: int = 3, hi: int = 12) -> list:
    """Batch of independent actuated lattice robots with a, b, c ~ U{lo..hi}."""
    rng = np.random.default_rng(seed)
    dims = rng.integers(lo, hi + 1, size=(n_robots, 3))
    return [actuated_box(int(a), int(b), int(c), rng) for a, b, c in dims]


def largest_component(occ: np.ndarray) -> np.ndarray:
    """Largest 26-connected component of a boolean voxel grid (nz, ny, nx)."""
    from scipy import ndimage
    lab, nlab = ndimage.label(occ, structure=np.ones((3, 3, 3), dtype=bool))
    if nlab == 0:
        return np.zeros_like(occ)
    sizes = np.bincount(lab.ravel())
    sizes[0] = 0
    return lab == int(np.argmax(sizes))


def voxel_morphology(rng: np.random.Generator, grid: int = 8, p: float = 0.6) -> np.ndarray:
    """Random voxel occupancy (nz, ny, nx): Bernoulli(p), largest component kept."""
    return largest_component(rng.random((grid, grid, grid)) < p)


def voxel_robot(occ: np.ndarray, phase_grid: np.ndarray, spacing: float = 0.1, mass: float = 0.1,
                k: float = 1e4, damping: float = 1.0, amp: float = 0.1, freq: float = 2.0) -> System:
    """Robot with one mass per occupied voxel and 26-neighbourhood springs.

    Each voxel v carries an actuation signal amp sin(2 pi f t + phi_v)
    (phase_grid is (nz, ny, nx), radians); a spring carries the mean of its two
    voxels' signals, amp cos((phi_i - phi_j) / 2) sin(2 pi f t + (phi_i +
    phi_j) / 2), so the rule does not depend on how voxels are numbered and a
    mirrored robot gets mirrored springs.
    """
    nz, ny, nx = occ.shape
    full_pos = lattice_points(nx, ny, nz, spacing)
    ends_full = lattice_springs(nx, ny, nz, occupied=occ)
    keep = np.flatnonzero(occ.ravel())
    remap = np.full(nx * ny * nz, -1, dtype=np.int64)
    remap[keep] = np.arange(keep.size)
    ends = remap[ends_full.astype(np.int64)].astype(np.uint32)
    pos = full_pos[keep]
    pos[:, 2] -= pos[:, 2].min()
    s = ends.shape[0]
    pi_ = phase_grid.ravel()[ends_full[:, 0].astype(np.int64)].astype(np.float64)
    pj_ = phase_grid.ravel()[ends_full[:, 1].astype(np.int64)].astype(np.float64)
    return System(pos=pos, vel=np.zeros_like(pos), mass=np.full(keep.size, mass),
                  fixed=np.zeros(keep.size, np.uint8), ends=ends, k=np.full(s, k),
                  rest=_initial_lengths(pos, ends), damping=np.full(s, damping), dt=1e-4,
                  ground=True, ground_k=1e5, mu=0.5, act_amp=amp * np.cos(0.5 * (pi_ - pj_)),
                  act_phase=0.5 * (pi_ + pj_), act_freq=freq, spacing=spacing, name="voxel_robot")


def two_masses(stretch: float = 1e-3, k: float = 1e4, m: float = 0.1, c: float = 0.0,
               length: float = 0.1, dt: float = 1e-5) -> System:
    """Two free masses joined by one spring stretched by ``stretch`` along x;
    no gravity, no ground."""
    pos = np.array([[0.0, 0.0, 0.0], [length + stretch, 0.0, 0.0]])
    return System(pos=pos, vel=np.zeros_like(pos), mass=np.array([m, m]),
                  fixed=np.zeros(2, np.uint8), ends=np.array([[0, 1]], np.uint32),
                  k=np.array([k]), rest=np.array([length]), damping=np.array([c]), dt=dt,
                  gravity=(0.0, 0.0, 0.0), ground=False, spacing=length, name="two_masses")


def material_stiffness(E: float, diameter: float, length: float) -> float:
    """Spring constant of a round bar of a real material (Sec. III-E, Eq. 2):
    k = E A_c / L_r with cross-section A_c = pi d^2 / 4."""
    return E * (np.pi * diameter * diameter / 4.0) / length

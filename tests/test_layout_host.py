"""Host-side layout builders (csrc/layout.cpp), checked on the CPU.

The step kernels trust these tables for every shared-memory and global index
they form, so the checks here are the bounds and consistency conditions the
kernels rely on: every spring appears once from each end, in the row of its
mass, pointing at its other end; on a grid every SELL column holds one cell
offset; every box-table read, padding included, lands inside its block's box
and on the slot of the intended neighbour; own and external slots are
distinct; and on a full lattice the box reads are free of shared-memory bank
conflicts.  layout.cpp is compiled here with the host compiler, through a
small C shim (tests/layout_shim.cpp).
"""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_1911_10274_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1911_10274_gb300", "csrc")
MAX_SLOTS = 1152
BLOCK = 256


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("no host C++ compiler")
    out = str(tmp_path_factory.mktemp("shim") / "liblayout_shim.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                    os.path.join(CSRC, "layout.cpp"), os.path.join(ROOT, "tests", "layout_shim.cpp"),
                    "-o", out], check=True)
    lib = C.CDLL(out)
    lib.shim_build.restype = C.c_int
    lib.shim_build.argtypes = [C.c_void_p, C.c_uint32, C.c_void_p, C.c_uint32, C.c_double, C.c_uint32]
    lib.shim_scalar.restype = C.c_uint64
    lib.shim_len.restype = C.c_uint64
    lib.shim_len.argtypes = [C.c_char_p]
    lib.shim_get.argtypes = [C.c_char_p, C.c_void_p]
    lib.shim_plan.restype = C.c_int
    lib.shim_plan.argtypes = [C.c_uint64, C.c_int, C.c_int]
    lib.shim_plan_scalar.restype = C.c_uint64
    lib.shim_records.argtypes = [C.c_uint32, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.shim_build_batch.restype = C.c_int
    lib.shim_build_batch.argtypes = [C.c_uint32, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.shim_batch_why.restype = C.c_char_p
    lib.shim_batch_scalar.restype = C.c_uint64
    lib.shim_batch_smem.restype = C.c_uint64
    lib.shim_batch_smem.argtypes = [C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, C.c_int]
    lib.shim_batch_len.restype = C.c_uint64
    lib.shim_batch_len.argtypes = [C.c_char_p]
    lib.shim_batch_get.argtypes = [C.c_char_p, C.c_void_p]
    return lib


class Layout:
    DT = {"caller_of_dev": np.uint32, "cell": np.int32, "slice_off": np.uint32, "nbr": np.uint32,
          "spring": np.uint32, "entry_of_end": np.uint32, "col_off": np.int16, "box_own_slot": np.uint16,
          "box_ext_off": np.uint32, "box_ext_idx": np.uint32, "box_ext_slot": np.uint16,
          "pslot": np.uint16, "phalo": np.uint32, "cube_base": np.uint32, "cube_meta": np.uint32,
          "cube_spring": np.uint32, "cube_pos_of_end": np.uint32, "box_dims": np.uint32}

    def __init__(self, lib, pos, ends):
        pos = np.ascontiguousarray(pos, np.float64)
        ends = np.ascontiguousarray(ends, np.uint32)
        d = np.linalg.norm(pos[ends[:, 1]] - pos[ends[:, 0]], axis=1)
        h = float(d[d > 0].min())
        assert lib.shim_build(pos.ctypes.data, len(pos), ends.ctypes.data, len(ends), h, MAX_SLOTS) == 0
        self.n, self.s = len(pos), len(ends)
        self.ends = ends
        self.n_dev, self.entries, self.grid, self.box_ok, self.halo_ok, self.box_slots, _, self.cube_ok, \
            self.cube_entries = [int(lib.shim_scalar(k)) for k in range(9)]
        for name, dt in self.DT.items():
            a = np.empty(int(lib.shim_len(name.encode())), dt)
            if a.size:
                lib.shim_get(name.encode(), a.ctypes.data)
            setattr(self, name, a)
        self.lib = lib
        self.dev_of = np.zeros(self.n, np.int64)
        real = self.caller_of_dev != np.uint32(0xFFFFFFFF)
        self.dev_of[self.caller_of_dev[real]] = np.nonzero(real)[0]

    def entry_coords(self):
        """(row mass, column index in the slice, global column) of every entry."""
        e = np.arange(self.entries, dtype=np.int64)
        sl = np.searchsorted(self.slice_off.astype(np.int64), e, side="right") - 1
        rel = e - self.slice_off[sl].astype(np.int64)
        return sl * 32 + rel % 32, rel // 32, self.slice_off[sl].astype(np.int64) // 32 + rel // 32


def lattice(nx, ny, nz, occupied=None):
    return inputs.lattice_points(nx, ny, nz, 0.1), inputs.lattice_springs(nx, ny, nz, occupied)


def check_sell(L):
    assert L.slice_off[0] == 0 and L.slice_off[-1] == L.entries
    assert np.all(np.diff(L.slice_off) % 64 == 0)                 # even widths of 32-entry columns
    real = L.spring != np.uint32(0xFFFFFFFF)
    assert real.sum() == 2 * L.s
    row, _, _ = L.entry_coords()
    # every spring once from each end, in its mass's row, pointing at the other end
    for end in (0, 1):
        e = L.entry_of_end[end::2].astype(np.int64)
        assert np.array_equal(L.spring[e], np.arange(L.s, dtype=np.uint32))
        assert np.array_equal(row[e], L.dev_of[L.ends[:, end]])
        assert np.array_equal(L.nbr[e], L.dev_of[L.ends[:, 1 - end]])
    pad = ~real
    assert np.array_equal(L.nbr[pad], np.where(row[pad] < L.n_dev, row[pad], 0))


def check_box(L):
    assert L.box_ok
    row, _, gcol = L.entry_coords()
    real = L.spring != np.uint32(0xFFFFFFFF)
    cell = L.cell.reshape(-1, 3).astype(np.int64)
    # columns are offset-aligned: one cell offset per (slice, column)
    off = cell[L.nbr[real]] - cell[row[real]]
    key = gcol[real]
    order = np.argsort(key, kind="stable")
    k_sorted, o_sorted = key[order], off[order]
    same = k_sorted[1:] == k_sorted[:-1]
    assert np.all(o_sorted[1:][same] == o_sorted[:-1][same])
    # slot arithmetic: own slot + column offset is the neighbour's slot in this block's box
    own = L.box_own_slot.astype(np.int64)
    holes = L.caller_of_dev == np.uint32(0xFFFFFFFF)
    assert np.all(own[holes] == 0xFFFF) and np.all(own[~holes] < L.box_slots)
    blk = row // BLOCK
    slot_of = {}
    n_blocks = (L.n_dev + BLOCK - 1) // BLOCK
    for b in range(n_blocks):
        m0, m1 = b * BLOCK, min(L.n_dev, (b + 1) * BLOCK)
        ext = L.box_ext_idx[L.box_ext_off[b]:L.box_ext_off[b + 1]].astype(np.int64)
        eslot = L.box_ext_slot[L.box_ext_off[b]:L.box_ext_off[b + 1]].astype(np.int64)
        mine = np.arange(m0, m1)[~holes[m0:m1]]
        slots = np.concatenate([own[mine], eslot])
        assert len(np.unique(slots)) == len(slots), f"block {b}: slots collide"
        assert slots.max() < L.box_slots and slots.min() >= 0
        assert not np.any((ext >= m0) & (ext < m1))
        slot_of[b] = dict(zip(np.concatenate([mine, ext]).tolist(), slots.tolist()))
    read = own[np.minimum(row, L.n_dev - 1)] + L.col_off[gcol].astype(np.int64)
    valid_row = (row < L.n_dev) & ~holes[np.minimum(row, L.n_dev - 1)]
    assert not np.any(real & ~valid_row)                       # holes carry no springs
    assert np.all(read[valid_row] >= 0) and np.all(read[valid_row] < L.box_slots)   # padding included
    for e in np.nonzero(real)[0]:
        assert read[e] == slot_of[blk[e]][int(L.nbr[e])]


def test_full_lattice_grid_layout_and_box_tables(shim):
    pos, ends = lattice(16, 16, 8)
    L = Layout(shim, pos, ends)
    assert L.grid and L.n_dev == L.n                            # 16 x 16 x 8 fills whole 8 x 8 x 4 cubes
    assert L.box_slots == 12 * 10 * 6                           # (8 + 2 -> 12) x (8 + 2) x (4 + 2)
    check_sell(L)
    check_box(L)
    # bank conflicts: per column, each quarter-warp's 16-byte reads hit 8 distinct
    # 16-byte bank groups, each half-warp's 8-byte reads 16 distinct 8-byte groups
    row, t, gcol = L.entry_coords()
    real = L.spring != np.uint32(0xFFFFFFFF)
    read = L.box_own_slot[row].astype(np.int64) + L.col_off[gcol].astype(np.int64)
    lane = row % 32
    bad = 0
    groups = 0
    for width, mod in ((8, 8), (16, 16)):
        gid = gcol * (32 // width) + lane // width
        for g in np.unique(gid):
            sel = (gid == g) & real
            if sel.sum() < width:
                continue                                          # boundary columns with padding
            groups += 1
            bad += len(np.unique(read[sel] % mod)) != width
    assert groups > 0 and bad == 0


def test_lattice_with_holes_and_second_neighbours(shim):
    pos, ends = lattice(10, 7, 5)
    idx = np.arange(10 * 7 * 5).reshape(5, 7, 10)
    far = np.stack([idx[:, :, :-2].ravel(), idx[:, :, 2:].ravel()], 1)
    dup = ends[:5]
    L = Layout(shim, pos, np.concatenate([ends, far, dup]))
    assert L.grid and L.n_dev > L.n                             # holes in partly filled cubes
    check_sell(L)
    check_box(L)


def test_voxel_robot_layout(shim):
    rng = np.random.default_rng(3)
    occ = inputs.voxel_morphology(rng)
    sys = inputs.voxel_robot(occ, rng.uniform(0, 2 * np.pi, occ.shape))
    L = Layout(shim, sys.pos, sys.ends)
    assert L.grid
    check_sell(L)
    check_box(L)


def test_unstructured_mesh_is_not_a_grid(shim):
    sys = inputs.random_mesh(n_points=2000, seed=5, lift=0.0)
    L = Layout(shim, sys.pos, sys.ends)
    assert not L.grid and not L.box_ok and L.n_dev == L.n
    check_sell(L)


def check_persistent_plan(L, smem_limit=220 * 1024):
    """Every row entry of a CTA reads either one of its own slots (the
    neighbour's index minus the CTA's first mass) or a halo slot whose halo
    entry names the neighbour's CTA and slot there; all reads stay inside the
    CTA's own + halo slots; the shared memory fits."""
    lib = L.lib
    if not lib.shim_plan(smem_limit, 0, 0):
        return False
    cl, per, threads, max_e, max_h, smem = [int(lib.shim_plan_scalar(k)) for k in range(6)]
    hoff = [int(lib.shim_plan_scalar(10 + r)) for r in range(9)]
    for name in ("pslot", "phalo"):
        a = np.empty(int(lib.shim_len(name.encode())), Layout.DT[name])
        if a.size:
            lib.shim_get(name.encode(), a.ctypes.data)
        setattr(L, name, a)
    assert cl in (1, 2, 4, 8) and per % 32 == 0 and cl * per >= L.n_dev and smem <= smem_limit
    assert threads == min(512, per)
    row, _, _ = L.entry_coords()
    for r in range(cl):
        m0, m1 = r * per, min(L.n_dev, (r + 1) * per)
        if m0 >= L.n_dev:
            break
        sel = (row >= m0) & (row < m1)
        nb = L.nbr[sel].astype(np.int64)
        sl = L.pslot[sel].astype(np.int64)
        halo = L.phalo[hoff[r]:hoff[r + 1]].astype(np.int64)
        assert len(halo) <= max_h and sel.sum() <= max_e
        own = (nb >= m0) & (nb < m1)
        assert np.array_equal(sl[own], nb[own] - m0)
        h = sl[~own] - per
        assert np.all(h >= 0) and np.all(h < len(halo))
        assert np.array_equal((halo[h] >> 16) * per + (halo[h] & 0xFFFF), nb[~own])
        assert len(np.unique(halo)) == len(halo)                        # each halo mass copied once
        assert not np.any(((halo >> 16) * per + (halo & 0xFFFF) >= m0) & ((halo >> 16) * per + (halo & 0xFFFF) < m1))
    return True


def test_persistent_plan_small_lattice_and_robot(shim):
    pos, ends = lattice(10, 10, 10)
    L = Layout(shim, pos, ends)
    assert check_persistent_plan(L)
    assert int(L.lib.shim_plan_scalar(1)) <= 512                          # one mass per thread
    rng = np.random.default_rng(8)
    occ = inputs.voxel_morphology(rng)
    sys = inputs.voxel_robot(occ, rng.uniform(0, 2 * np.pi, occ.shape))
    assert check_persistent_plan(Layout(shim, sys.pos, sys.ends))
    mesh = inputs.random_mesh(n_points=1500, seed=6, lift=0.0)
    assert check_persistent_plan(Layout(shim, mesh.pos, mesh.ends))


def test_persistent_plan_refuses_what_does_not_fit(shim):
    pos, ends = lattice(20, 20, 20)
    L = Layout(shim, pos, ends)
    assert not L.lib.shim_plan(220 * 1024, 0, 0)


CUBE_DIRS = [(1, 0, 0), (-1, 1, 0), (0, 1, 0), (1, 1, 0), (-1, -1, 1), (0, -1, 1), (1, -1, 1),
             (-1, 0, 1), (0, 0, 1), (1, 0, 1), (-1, 1, 1), (0, 1, 1), (1, 1, 1)]


def check_cube(L):
    """Replays the cube kernel's data flow on the host: for every mass, the
    springs it adds in pass order (+p from its plus entry, then -p received
    from the in-cube partner's plus entry or read from the ext stream) are
    exactly its SELL row, in order; every spring end is stored once or
    received; the pass offsets match the box geometry."""
    assert L.cube_ok
    NONE = 0xFFFFFFFF
    P, W = 13, 8
    cell = L.cell.reshape(-1, 3).astype(np.int64)
    dev_of_cell = {tuple(c): d for d, c in enumerate(cell.tolist())}
    meta = L.cube_meta.reshape(-1, P, W, 4)
    dims = L.box_dims.reshape(-1, 2).astype(np.int64)
    row, _, _ = L.entry_coords()
    real = L.spring != NONE
    order = np.argsort(row[real], kind="stable")
    rows = {}
    for m, q in zip(row[real][order].tolist(), L.spring[real][order].tolist()):
        rows.setdefault(m, []).append(q)
    n_cubes = L.n_dev // BLOCK
    assert len(L.cube_base) == n_cubes + 1 and np.all(L.cube_base[:-1] % 16 == 0)
    for b in range(n_cubes):
        base = int(L.cube_base[b])
        ext0 = base + P * BLOCK
        for j, (dx, dy, dz) in enumerate(CUBE_DIRS):
            off = np.int16(meta[b, j, 0, 3] & 0xFFFF)
            assert off == dx + dims[b, 0] * dy + dims[b, 0] * dims[b, 1] * dz
        for t in range(BLOCK):
            m = b * BLOCK + t
            w, l = divmod(t, 32)
            seq = []
            for j, (dx, dy, dz) in enumerate(CUBE_DIRS):
                q = int(L.cube_spring[base + j * BLOCK + t])
                if q != NONE:
                    seq.append(q)
                recv, ext, ebase = int(meta[b, j, w, 0]), int(meta[b, j, w, 1]), int(meta[b, j, w, 2])
                assert not (recv >> l & 1 and ext >> l & 1)
                if recv >> l & 1:
                    pm = dev_of_cell[(cell[m, 0] - dx, cell[m, 1] - dy, cell[m, 2] - dz)]
                    assert b * BLOCK <= pm < (b + 1) * BLOCK
                    seq.append(int(L.cube_spring[base + j * BLOCK + (pm - b * BLOCK)]))
                elif ext >> l & 1:
                    seq.append(int(L.cube_spring[ext0 + ebase + bin(ext & ((1 << l) - 1)).count("1")]))
            assert seq == rows.get(m, []), (m, seq, rows.get(m))
    # every spring: one end at a plus entry, the other at an ext entry or received
    pe = L.cube_pos_of_end.reshape(-1, 2)
    stored = (pe != NONE).sum(1)
    assert np.all(stored >= 1) and np.all(stored <= 2)
    for q, (a, c) in enumerate(pe.tolist()):
        for pos in (a, c):
            if pos != NONE:
                assert L.cube_spring[pos] == q


def test_cube_layout_replays_every_row_in_order(shim):
    pos, ends = lattice(16, 16, 8)
    L = Layout(shim, pos, ends)
    check_cube(L)
    # springs inside a cube are stored once: fewer entries than half-edges
    assert L.cube_entries < 0.75 * 2 * L.s


def test_cube_layout_with_holes(shim):
    pos, ends = lattice(10, 7, 5)
    L = Layout(shim, pos, ends)
    check_cube(L)
    rng = np.random.default_rng(3)
    occ = inputs.voxel_morphology(rng)
    sys = inputs.voxel_robot(occ, rng.uniform(0, 2 * np.pi, occ.shape))
    check_cube(Layout(shim, sys.pos, sys.ends))


def test_cube_layout_refuses_second_neighbours_and_duplicates(shim):
    pos, ends = lattice(10, 7, 5)
    idx = np.arange(10 * 7 * 5).reshape(5, 7, 10)
    far = np.stack([idx[:, :, :-2].ravel(), idx[:, :, 2:].ravel()], 1)
    assert not Layout(shim, pos, np.concatenate([ends, far])).cube_ok
    assert not Layout(shim, pos, np.concatenate([ends, ends[:3]])).cube_ok


# ---------------------------------------------------------------- batch layout

class BatchLayout:
    """titan_batch_create's host layout of a list of inputs.System, read back
    through the shim."""
    CTA_FIELDS = ("mass_begin", "mass_count", "slot_count", "edge_off", "edge_count", "slice_base", "n_slices",
                  "robot", "halo_off", "halo_count", "halo_slots")
    DT = {"ctas": np.uint32, "groups": np.uint64, "slices": np.uint32, "kl": np.float32, "act": np.float32,
          "nbr": np.uint16, "halo": np.uint32, "mass_off": np.uint32, "mass_cnt": np.uint32, "mass_of_slot": np.uint32,
          "init_state": np.float32}

    def __init__(self, lib, systems):
        from paper_1911_10274_gb300 import titan as T
        keep, ms, ss, acts = [], [], [], []
        for sy in systems:
            d = dict(pos=np.ascontiguousarray(sy.pos, np.float64), vel=np.ascontiguousarray(sy.vel, np.float64),
                     mass=np.ascontiguousarray(sy.mass, np.float64), fixed=np.ascontiguousarray(sy.fixed, np.uint8),
                     ends=np.ascontiguousarray(sy.ends, np.uint32), k=np.ascontiguousarray(sy.k, np.float64),
                     rest=np.ascontiguousarray(sy.rest, np.float64))
            ptr = lambda a: a.ctypes.data if a.size else None
            ms.append(T.titan_masses(sy.n_masses, ptr(d["pos"]), ptr(d["vel"]), ptr(d["mass"]), ptr(d["fixed"])))
            ss.append(T.titan_springs(sy.n_springs, ptr(d["ends"]), ptr(d["k"]), ptr(d["rest"]), None))
            if sy.act_amp is not None:
                d["amp"] = np.ascontiguousarray(sy.act_amp, np.float64)
                d["phase"] = np.ascontiguousarray(sy.act_phase, np.float64)
                acts.append(T.titan_actuation(ptr(d["amp"]), ptr(d["phase"]), float(sy.act_freq)))
            else:
                acts.append(T.titan_actuation(None, None, 0.0))
            keep.append(d)
        n = len(systems)
        M = (T.titan_masses * max(1, n))(*ms)
        S = (T.titan_springs * max(1, n))(*ss)
        A = (T.titan_actuation * max(1, n))(*acts)
        self.ok = lib.shim_build_batch(n, C.addressof(M), C.addressof(S), C.addressof(A)) == 1
        self.why = lib.shim_batch_why().decode()
        if not self.ok:
            return
        self.total_slots, self.any_act = int(lib.shim_batch_scalar(0)), bool(lib.shim_batch_scalar(1))
        for name, dt in self.DT.items():
            a = np.empty(int(lib.shim_batch_len(name.encode())), dt)
            if a.size:
                lib.shim_batch_get(name.encode(), a.ctypes.data)
            setattr(self, name, a)
        self.ctas = self.ctas.reshape(-1, 11).astype(np.int64)
        self.groups = self.groups.reshape(-1, 4).astype(np.int64)
        self.kl = self.kl.reshape(-1, 2)
        self.act = self.act.reshape(-1, 2)
        self.init_state = self.init_state.reshape(-1, 8)
        self.cta = [dict(zip(self.CTA_FIELDS, row)) for row in self.ctas]


def _batch_systems():
    """Robots of every cluster size and shared-memory class, plus the
    degenerate systems: one spring, no springs, fixed masses with velocities,
    an unactuated system among actuated ones."""
    rng = np.random.default_rng(5)
    out = [inputs.actuated_box(a, b, c, rng) for a, b, c in
           [(3, 3, 3), (12, 12, 12), (5, 4, 3), (14, 14, 14), (7, 3, 9), (10, 10, 10), (8, 8, 8), (4, 11, 6),
            (3, 12, 3), (9, 9, 9)]]
    two = inputs.two_masses()
    two.act_amp, two.act_phase = None, None
    out.append(two)
    lone = inputs.actuated_box(2, 1, 1, rng)
    lone.ends = np.zeros((0, 2), np.uint32)
    for f in ("k", "rest", "damping"):
        setattr(lone, f, np.zeros(0))
    lone.act_amp, lone.act_phase = None, None
    out.append(lone)
    fx = inputs.actuated_box(6, 5, 4, rng)
    fx.fixed[:30] = 1
    fx.vel[:] = rng.normal(0.0, 0.1, fx.vel.shape)
    out.append(fx)
    plain = inputs.actuated_box(9, 8, 7, rng)
    plain.act_amp, plain.act_phase = None, None
    out.append(plain)
    return out


def _decode_slot(L, c, rank, P, slot, base):
    """Caller index (within its system) of the mass a table slot names
    (base: the system's first global slot); -1 for a padding slot."""
    own = slot < P
    g = np.where(own, rank * P + slot.astype(np.int64), 0)
    if (~own).any():
        code = L.halo[c["halo_off"] + slot[~own].astype(np.int64) - P].astype(np.int64)
        g[~own] = (code >> 16) * P + (code & 0xFFFF)
    j = L.mass_of_slot[base + g].astype(np.int64)
    return np.where(j == 0xFFFFFFFF, -1, j)


def test_batch_layout_encodes_every_spring_and_every_index_stays_in_range(shim):
    systems = _batch_systems()
    L = BatchLayout(shim, systems)
    assert L.ok, L.why
    E = L.nbr.size
    assert L.kl.shape[0] == E and (not L.any_act or L.act.shape[0] == E)
    # groups: consecutive, cover every CTA, whole clusters, cluster sizes non-increasing
    assert L.groups[0, 1] == 0 and L.groups[-1, 1] + L.groups[-1, 2] == len(L.cta)
    assert np.all(L.groups[1:, 1] == L.groups[:-1, 1] + L.groups[:-1, 2])
    assert np.all(L.groups[:, 2] % L.groups[:, 0] == 0) and np.all(np.diff(L.groups[:, 0]) <= 0)
    assert set(L.groups[:, 0]) == {1, 2, 4, 8}
    # incidence of every system: springs of mass i = inc[r][inc_ptr[r][i]:inc_ptr[r][i + 1]]
    inc, inc_ptr = [], []
    for sy in systems:
        half = np.concatenate([sy.ends[:, 0], sy.ends[:, 1]]).astype(np.int64)
        spr = np.concatenate([np.arange(sy.n_springs)] * 2)
        o = np.argsort(half, kind="stable")
        inc.append(spr[o])
        inc_ptr.append(np.searchsorted(half[o], np.arange(sy.n_masses + 1)))
    seen_robots = []
    for cluster, first, count, smem in L.groups:
        assert smem <= 220 * 1024
        for c0 in range(first, first + count, cluster):
            cl = L.cta[c0:c0 + cluster]
            r = cl[0]["robot"]
            sy = systems[r]
            n = sy.n_masses
            seen_robots.append(r)
            P = cl[0]["slot_count"]
            assert P % 32 == 0 and P <= 4096 and cluster * P >= n
            for rank, c in enumerate(cl):
                # one system and one state layout per cluster, CTA q at rank q
                assert c["robot"] == r and c["slot_count"] == P
                assert c["halo_slots"] == max(x["halo_count"] for x in cl)
                m0, m1 = min(n, rank * P), min(n, rank * P + P)
                assert c["mass_begin"] == L.mass_off[r] + m0 and c["mass_count"] == m1 - m0
                assert c["mass_begin"] + P <= L.total_slots
                # every array range the bulk copies and the kernel read
                assert c["n_slices"] * 32 == P and c["slice_base"] % 4 == 0
                assert c["slice_base"] + (c["n_slices"] + 4) // 4 * 4 <= L.slices.size
                assert c["edge_off"] % 64 == 0 and c["edge_count"] % 64 == 0
                assert c["edge_off"] + c["edge_count"] <= E
                assert c["halo_off"] + c["halo_count"] <= L.halo.size
                assert shim.shim_batch_smem(P, c["halo_slots"], c["n_slices"], c["edge_count"],
                                            int(L.any_act)) <= smem
                # slots: the CTA's own masses (caller range [m0, m1)) by decreasing degree, padding after
                base = L.mass_off[r]
                ms = L.mass_of_slot[base + rank * P:base + rank * P + P].astype(np.int64)
                real = ms[:m1 - m0]
                assert np.array_equal(np.sort(real), np.arange(m0, m1)) and np.all(ms[m1 - m0:] == 0xFFFFFFFF)
                dg = np.diff(inc_ptr[r])
                assert np.all(np.diff(dg[real]) <= 0)
                # halo: other ranks of this cluster, masses that exist, no repeats
                hl = L.halo[c["halo_off"]:c["halo_off"] + c["halo_count"]].astype(np.int64)
                hr, hs = hl >> 16, hl & 0xFFFF
                assert np.all(hr < cluster) and np.all(hr != rank) and np.all(hs < P)
                assert np.all(L.mass_of_slot[base + hr * P + hs] < n) and len(set(hl.tolist())) == hl.size
                rel = L.slices[c["slice_base"]:c["slice_base"] + c["n_slices"] + 1].astype(np.int64)
                assert rel[0] == 0 and np.all(np.diff(rel) % 64 == 0) and rel[-1] <= c["edge_count"]
                nb = L.nbr[c["edge_off"]:c["edge_off"] + c["edge_count"]]
                kl = L.kl[c["edge_off"]:c["edge_off"] + c["edge_count"]]
                ac = L.act[c["edge_off"]:c["edge_off"] + c["edge_count"]] if L.any_act else None
                assert np.all(nb[:rel[-1]] < P + c["halo_count"])
                # rows: decode each lane's entries back to (neighbour, k, L0) and compare with the springs
                got = {}
                for s_ in range(c["n_slices"]):
                    w = (rel[s_ + 1] - rel[s_]) // 32
                    for lane in range(32):
                        p_ = s_ * 32 + lane                               # the row's slot
                        i = int(ms[p_]) if p_ < m1 - m0 else -1           # caller index of its mass
                        e = rel[s_] + 32 * np.arange(w) + lane
                        j = _decode_slot(L, c, rank, P, nb[e], base)
                        pad = (kl[e, 0] == 0) & (kl[e, 1] == 0)
                        assert np.all(nb[e][pad] == p_), (r, i)           # padding names the row's own slot
                        if i < 0:
                            assert pad.all()
                            continue
                        assert not pad[:np.count_nonzero(~pad)].any()  # springs first, padding after
                        got[i] = (j[~pad], kl[e][~pad], None if ac is None else ac[e][~pad])
                for i, (j, k, a) in got.items():
                    q = inc[r][inc_ptr[r][i]:inc_ptr[r][i + 1]]
                    other = np.where(sy.ends[q, 0] == i, sy.ends[q, 1], sy.ends[q, 0]).astype(np.int64)
                    order = np.lexsort((q, other))                       # by (neighbour, spring)
                    q, other = q[order], other[order]
                    assert np.array_equal(j, other), (r, i)
                    assert np.array_equal(k[:, 0], sy.k[q].astype(np.float32))
                    assert np.array_equal(k[:, 1], sy.rest[q].astype(np.float32))
                    if a is not None:
                        if sy.act_amp is None:
                            assert not a.any()
                        else:
                            A, ph = sy.act_amp[q], sy.act_phase[q]
                            np.testing.assert_array_equal(a[:, 0], (A * np.cos(ph)).astype(np.float32))
                            np.testing.assert_array_equal(a[:, 1], (A * np.sin(ph)).astype(np.float32))
            # initial state: every real mass in its slot (the first n slots), padding slots fixed and at rest
            st = L.init_state[L.mass_off[r]:L.mass_off[r] + cluster * P]
            who = L.mass_of_slot[L.mass_off[r]:L.mass_off[r] + n].astype(np.int64)
            assert np.array_equal(np.sort(who), np.arange(n))
            assert np.array_equal(st[:n, :3], sy.pos[who].astype(np.float32))
            assert np.array_equal(st[:n, 4:7], sy.vel[who].astype(np.float32))
            inv = np.where(sy.fixed.astype(bool), 0.0, 1.0 / sy.mass).astype(np.float32)
            assert np.array_equal(st[:n, 3], inv[who]) and not st[n:].any() and not st[:, 7].any()
    assert sorted(seen_robots) == list(range(len(systems)))
    assert L.total_slots == L.init_state.shape[0]


def test_batch_layout_refuses_a_system_too_dense_for_a_cluster(shim):
    """4096 masses each joined to its 32 successors: 64 half-edges per mass do
    not fit 8 CTAs of 220 KB; the builder says which system."""
    small = inputs.actuated_box(3, 3, 3, np.random.default_rng(0))
    n, reach = 4096, 32
    pos = np.zeros((n, 3))
    pos[:, 0] = 0.1 * np.arange(n)
    ends = np.array([(i, i + d) for i in range(n) for d in range(1, reach + 1) if i + d < n], np.uint32)
    s = ends.shape[0]
    dense = inputs.System(pos=pos, vel=np.zeros_like(pos), mass=np.full(n, 0.1), fixed=np.zeros(n, np.uint8),
                          ends=ends, k=np.full(s, 1e3), rest=0.1 * (ends[:, 1] - ends[:, 0]).astype(np.float64),
                          damping=np.full(s, 1.0), dt=1e-4)
    L = BatchLayout(shim, [small, dense])
    assert not L.ok and L.why == "system 1 does not fit a cluster of 8 CTAs"
    assert BatchLayout(shim, [small]).ok


def test_spring_records_are_sorted_by_device_ends_and_stable(shim):
    """The atomic path's records: a permutation of the springs sorted by
    (lower, higher) device index of their ends, duplicate springs kept in
    caller order, with slot_of_spring its inverse."""
    sy = inputs.random_mesh(n_points=3000, knn=6, seed=4)
    ends = np.concatenate([sy.ends, sy.ends[:50][:, ::-1], sy.ends[10:20]]).astype(np.uint32)   # duplicates, both orientations
    ends = np.ascontiguousarray(ends)
    L = Layout(shim, sy.pos, ends)
    s = len(ends)
    order = np.empty(s, np.uint32)
    slot = np.empty(s, np.uint32)
    shim.shim_records(s, ends.ctypes.data, order.ctypes.data, slot.ctypes.data)
    assert np.array_equal(np.sort(order), np.arange(s))
    assert np.array_equal(slot[order], np.arange(s))
    d = L.dev_of[ends.astype(np.int64)]
    lo, hi = d.min(axis=1), d.max(axis=1)
    key = lo[order] * (1 << 32) + hi[order]
    assert np.all(np.diff(key) >= 0)
    tie = np.diff(key) == 0
    assert np.all(np.diff(order.astype(np.int64))[tie] > 0)     # equal keys stay in caller order

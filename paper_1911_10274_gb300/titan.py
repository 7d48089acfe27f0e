"""Thin ctypes binding of libtitan.so (include/titan.h).

Functions carry the C names and only marshal arguments: numpy arrays become
host pointers, torch CUDA tensors and streams become device pointers and
cudaStream_t handles.  Every step of the simulation runs in the library's
CUDA kernels; there is no Python or CPU fallback - if the library cannot be
built or loaded, loading fails with an error.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Optional

import numpy as np

from . import build as _build

TITAN_OK, TITAN_E_INVALID, TITAN_E_CUDA, TITAN_E_OOM, TITAN_E_TIMEOUT, TITAN_E_BUSY, \
    TITAN_E_UNSUPPORTED = range(7)
ACCUM_CSR, ACCUM_ATOMIC = 0, 1
ORDER_INPUT, ORDER_MORTON = 0, 1
EXEC_AUTO, EXEC_LAUNCH, EXEC_PERSISTENT = 0, 1, 2
_STATUS = {0: "TITAN_OK", 1: "TITAN_E_INVALID", 2: "TITAN_E_CUDA", 3: "TITAN_E_OOM",
           4: "TITAN_E_TIMEOUT", 5: "TITAN_E_BUSY", 6: "TITAN_E_UNSUPPORTED"}


class TitanError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


class titan_masses(C.Structure):
    _fields_ = [("n", C.c_uint32), ("pos", C.c_void_p), ("vel", C.c_void_p),
                ("mass", C.c_void_p), ("fixed", C.c_void_p)]


class titan_springs(C.Structure):
    _fields_ = [("n", C.c_uint32), ("ends", C.c_void_p), ("k", C.c_void_p),
                ("rest", C.c_void_p), ("damping", C.c_void_p)]


class titan_params(C.Structure):
    _fields_ = [("dt", C.c_double), ("gravity", C.c_double * 3), ("ground", C.c_int32),
                ("ground_k", C.c_double), ("mu", C.c_double), ("damping", C.c_double),
                ("accumulate", C.c_int32), ("order", C.c_int32), ("exec", C.c_int32),
                ("device", C.c_int32), ("stream", C.c_void_p), ("spin_limit", C.c_uint64),
                ("graph_chunk", C.c_int32), ("kernel_variant", C.c_int32),
                ("l2_persist", C.c_int32), ("launch_overlap", C.c_int32), ("reserved", C.c_int32 * 4)]


class titan_actuation(C.Structure):
    _fields_ = [("amp", C.c_void_p), ("phase", C.c_void_p), ("freq_hz", C.c_double)]


_lib = None
_lock = threading.Lock()
_P = C.c_void_p


def load(path: Optional[str] = None):
    """Builds (if stale) and loads libtitan.so; raises if that is impossible."""
    global _lib
    with _lock:
        if _lib is None:
            lib_path = path or _build.build()
            lib = C.CDLL(lib_path)
            S, u32, u64, f32 = C.c_int, C.c_uint32, C.c_uint64, C.c_float
            sigs = {
                "titan_default_params": (None, [C.POINTER(titan_params)]),
                "titan_create": (S, [C.POINTER(titan_masses), C.POINTER(titan_springs),
                                     C.POINTER(titan_params), C.POINTER(_P)]),
                "titan_step": (S, [_P, u64]),
                "titan_snapshot_async": (S, [_P, _P, C.POINTER(u64)]),
                "titan_snapshot_wait": (S, [_P, u64, C.POINTER(C.POINTER(f32)),
                                            C.POINTER(C.POINTER(f32)), C.POINTER(C.c_double)]),
                "titan_set_actuation": (S, [_P, u32, _P, _P, _P, f32]),
                "titan_set_actuation_dev": (S, [_P, u32, _P, _P, f32]),
                "titan_group_centroids": (S, [_P, u32, _P, _P, _P]),
                "titan_group_seed": (S, [_P, u32, _P, _P, C.c_int32, _P]),
                "titan_set_state": (S, [_P, _P, _P]),
                "titan_read_state_dev": (S, [_P, _P, _P, _P]),
                "titan_sync": (S, [_P]),
                "titan_steps": (u64, [_P]),
                "titan_csr_kernel": (C.c_int32, [_P]),
                "titan_exec_mode": (C.c_int32, [_P]),
                "titan_last_error": (C.c_char_p, [_P]),
                "titan_destroy": (S, [_P]),
                "titan_step_atomic_noalloc": (S, [u32, _P, _P, _P, u32, _P, _P, _P, f32,
                                                  C.POINTER(titan_params), _P, _P, _P]),
                "titan_set_step": (S, [_P, u64]),
                "titan_selftest_wait_timeout": (S, [C.c_int32, u32]),
                "titan_set_worm_actuation": (S, [_P, u32, _P, _P, _P, f32, f32]),
                "titan_set_spring_params": (S, [_P, u32, _P, _P, _P, _P]),
                "titan_remove_springs": (S, [_P, u32, _P]),
                "titan_add_springs": (S, [_P, u32, _P, _P, _P, _P, C.POINTER(u32)]),
                "titan_add_masses": (S, [_P, u32, _P, _P, _P, _P, C.POINTER(u32)]),
                "titan_set_fixed": (S, [_P, u32, _P, _P]),
                "titan_adjoint": (S, [_P, u64, u32, _P, _P, _P, _P]),
                "titan_gemm_bf16_tn": (S, [u32, u32, u32, _P, _P, _P, _P]),
                "titan_gemm_check": (S, []),
                "titan_mlp_create": (S, [u32, u32, u64, C.c_int32, _P, C.POINTER(_P)]),
                "titan_mlp_param_count": (u64, [_P]),
                "titan_mlp_get_params": (S, [_P, _P]),
                "titan_mlp_set_params": (S, [_P, _P]),
                "titan_mlp_forward": (S, [_P, _P, u32, _P]),
                "titan_mlp_gradient": (S, [_P, _P, _P, u32, _P, _P]),
                "titan_mlp_train_step": (S, [_P, _P, _P, u32, f32, _P]),
                "titan_mlp_sync": (S, [_P]),
                "titan_mlp_last_error": (C.c_char_p, [_P]),
                "titan_mlp_destroy": (S, [_P]),
                "titan_batch_create": (S, [u32, C.POINTER(titan_masses), C.POINTER(titan_springs),
                                           C.POINTER(titan_actuation), C.POINTER(titan_params),
                                           C.POINTER(_P)]),
                "titan_batch_rollout": (S, [_P, u64]),
                "titan_batch_autotune": (S, [_P, u32]),
                "titan_batch_reset": (S, [_P]),
                "titan_batch_sync": (S, [_P]),
                "titan_batch_read": (S, [_P, u32, _P, _P]),
                "titan_batch_centroids": (S, [_P, _P]),
                "titan_batch_groups": (u32, [_P]),
                "titan_batch_system_group": (S, [_P, u32, C.POINTER(u32)]),
                "titan_batch_configure": (S, [_P, u32, u32, u32]),
                "titan_batch_info": (S, [_P, u32, C.POINTER(u32), C.POINTER(u32), C.POINTER(u32), C.POINTER(u32)]),
                "titan_batch_last_error": (C.c_char_p, [_P]),
                "titan_batch_destroy": (S, [_P]),
            }
            for name, (res, args) in sigs.items():
                fn = getattr(lib, name)
                fn.restype, fn.argtypes = res, args
            _lib = lib
    return _lib


def _check(status: int, sim=None):
    if status != TITAN_OK:
        msg = load().titan_last_error(sim).decode(errors="replace")
        raise TitanError(status, msg)


def _ptr(a) -> Optional[int]:
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


# --------------------------------------------------------------------------- C names

def titan_default_params() -> titan_params:
    p = titan_params()
    load().titan_default_params(C.byref(p))
    return p


def titan_create(masses: titan_masses, springs: titan_springs, params: titan_params) -> int:
    out = _P()
    _check(load().titan_create(C.byref(masses), C.byref(springs), C.byref(params), C.byref(out)))
    return out.value


def titan_step(sim: int, n_steps: int) -> None:
    _check(load().titan_step(sim, n_steps), sim)


def titan_snapshot_async(sim: int, stream: Optional[int] = None) -> int:
    t = C.c_uint64()
    _check(load().titan_snapshot_async(sim, stream, C.byref(t)), sim)
    return t.value


def titan_snapshot_wait(sim: int, ticket: int, n: int, copy: bool = True):
    """Returns (pos, vel, t): pos/vel [n][3] float32, numpy copies, or with
    copy=False read-only views of the library's pinned snapshot buffers (no
    host copy; valid until the second next titan_snapshot_async)."""
    p, v, t = C.POINTER(C.c_float)(), C.POINTER(C.c_float)(), C.c_double()
    _check(load().titan_snapshot_wait(sim, ticket, C.byref(p), C.byref(v), C.byref(t)), sim)
    if n == 0:
        return np.zeros((0, 3), np.float32), np.zeros((0, 3), np.float32), t.value
    pos = np.ctypeslib.as_array(p, shape=(n, 3))
    vel = np.ctypeslib.as_array(v, shape=(n, 3))
    if copy:
        return pos.copy(), vel.copy(), t.value
    pos.flags.writeable = False
    vel.flags.writeable = False
    return pos, vel, t.value


def titan_set_actuation(sim: int, spring_ids, amp, phase, freq_hz: float) -> None:
    ids = np.ascontiguousarray(spring_ids, dtype=np.uint32)
    a = np.ascontiguousarray(amp, dtype=np.float32)
    ph = np.ascontiguousarray(phase, dtype=np.float32)
    if not (ids.shape == a.shape == ph.shape):
        raise ValueError("spring_ids, amp and phase must have the same length")
    _check(load().titan_set_actuation(sim, ids.size, _ptr(ids), _ptr(a), _ptr(ph), float(freq_hz)), sim)


def titan_set_actuation_dev(sim: int, amp_dev, phase_dev, freq_hz: float) -> None:
    """Every spring's (amp, phase) from 1-D contiguous CUDA float32 tensors
    of n_springs entries each (caller order), copied on the simulation's
    stream; the library checks the length against its spring count."""
    import torch
    for name, t in (("amp_dev", amp_dev), ("phase_dev", phase_dev)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32:
            raise TypeError(f"titan_set_actuation_dev: {name} must be a CUDA float32 tensor")
        if t.dim() != 1 or not t.is_contiguous():
            raise ValueError(f"titan_set_actuation_dev: {name} must be 1-D and contiguous")
    if amp_dev.numel() != phase_dev.numel():
        raise ValueError("titan_set_actuation_dev: amp_dev and phase_dev must have the same length")
    _check(load().titan_set_actuation_dev(sim, amp_dev.numel(), _ptr(amp_dev), _ptr(phase_dev), float(freq_hz)),
           sim)


def titan_group_centroids(sim: int, first_dev, origin_dev, out_dev) -> None:
    """out_dev[g] = mean position of masses first_dev[g] .. first_dev[g+1]-1
    (minus origin_dev[g] if given); CUDA tensors: uint32/int32 [G+1], float32
    [G][3]; enqueued on the simulation's stream."""
    _check(load().titan_group_centroids(sim, first_dev.numel() - 1, _ptr(first_dev), _ptr(origin_dev),
                                        _ptr(out_dev)), sim)


def titan_group_seed(sim: int, first_dev, w_dev, axis: int, seed_dev) -> None:
    """seed_dev[i][axis] = w_dev[g] / |group g| for the masses of group g, 0
    elsewhere; enqueued on the simulation's stream."""
    _check(load().titan_group_seed(sim, first_dev.numel() - 1, _ptr(first_dev), _ptr(w_dev), int(axis),
                                   _ptr(seed_dev)), sim)


def titan_set_state(sim: int, pos, vel=None) -> None:
    p = np.ascontiguousarray(pos, dtype=np.float64)
    v = None if vel is None else np.ascontiguousarray(vel, dtype=np.float64)
    _check(load().titan_set_state(sim, _ptr(p), _ptr(v)), sim)


def titan_read_state_dev(sim: int, pos_dev=None, vel_dev=None, stream: Optional[int] = None) -> None:
    _check(load().titan_read_state_dev(sim, _ptr(pos_dev), _ptr(vel_dev), stream), sim)


def _u32(a):
    return np.ascontiguousarray(a, dtype=np.uint32)


def _f64opt(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def titan_set_worm_actuation(sim: int, spring_ids, c, t_offset, omega: float, period: float) -> None:
    ids, cc = _u32(spring_ids), np.ascontiguousarray(c, np.float32)
    to = np.ascontiguousarray(t_offset, np.float32)
    _check(load().titan_set_worm_actuation(sim, ids.size, _ptr(ids), _ptr(cc), _ptr(to), float(omega), float(period)), sim)


def titan_set_spring_params(sim: int, spring_ids, k=None, rest=None, damping=None) -> None:
    ids = _u32(spring_ids)
    k, rest, damping = _f64opt(k), _f64opt(rest), _f64opt(damping)
    _check(load().titan_set_spring_params(sim, ids.size, _ptr(ids), _ptr(k), _ptr(rest), _ptr(damping)), sim)


def titan_remove_springs(sim: int, spring_ids) -> None:
    ids = _u32(spring_ids)
    _check(load().titan_remove_springs(sim, ids.size, _ptr(ids)), sim)


def titan_add_springs(sim: int, ends, k, rest=None, damping=None) -> int:
    e = _u32(ends).reshape(-1)
    k, rest, damping = _f64opt(k), _f64opt(rest), _f64opt(damping)
    first = C.c_uint32()
    _check(load().titan_add_springs(sim, e.size // 2, _ptr(e), _ptr(k), _ptr(rest), _ptr(damping), C.byref(first)), sim)
    return first.value


def titan_add_masses(sim: int, pos, mass, vel=None, fixed=None) -> int:
    p, m = _f64opt(pos).reshape(-1), _f64opt(mass)
    v = None if vel is None else _f64opt(vel).reshape(-1)
    f = None if fixed is None else np.ascontiguousarray(fixed, np.uint8)
    first = C.c_uint32()
    _check(load().titan_add_masses(sim, m.size, _ptr(p), _ptr(v), _ptr(m), _ptr(f), C.byref(first)), sim)
    return first.value


def titan_set_fixed(sim: int, mass_ids, fixed) -> None:
    ids = _u32(mass_ids)
    f = np.ascontiguousarray(fixed, np.uint8)
    _check(load().titan_set_fixed(sim, ids.size, _ptr(ids), _ptr(f)), sim)


def titan_set_step(sim: int, step: int) -> None:
    _check(load().titan_set_step(sim, step), sim)


def titan_adjoint(sim: int, n_steps: int, every: int, seed_pos_dev, seed_vel_dev, grad_amp_dev,
                  grad_phase_dev) -> None:
    _check(load().titan_adjoint(sim, n_steps, every, _ptr(seed_pos_dev), _ptr(seed_vel_dev),
                                _ptr(grad_amp_dev), _ptr(grad_phase_dev)), sim)


def titan_sync(sim: int) -> None:
    _check(load().titan_sync(sim), sim)


def titan_steps(sim: int) -> int:
    return int(load().titan_steps(sim))


def titan_last_error(sim: Optional[int] = None) -> str:
    return load().titan_last_error(sim).decode(errors="replace")


def titan_destroy(sim: int) -> None:
    _check(load().titan_destroy(sim))


def check_noalloc_args(n_masses: int, n_springs: int, pos, vel, inv_mass, ends, k, rest, pos_out, vel_out,
                       device=None) -> None:
    """Checks the tensors of titan_step_atomic_noalloc before anything is
    launched: the C call takes raw device pointers, so a host array, a tensor
    of the wrong type, size or device, or an output that shares memory with an
    input would otherwise be read or written blindly.  `device` is the device
    the tensors must be on (default: the current CUDA device).  Raises
    TypeError or ValueError."""
    import torch
    if device is None:
        device = torch.device("cuda", torch.cuda.current_device())
    named = dict(pos=pos, vel=vel, inv_mass=inv_mass, ends=ends, k=k, rest=rest, pos_out=pos_out,
                 vel_out=vel_out)
    sizes = dict(pos=3 * n_masses, vel=3 * n_masses, inv_mass=n_masses, ends=2 * n_springs, k=n_springs,
                 rest=n_springs, pos_out=3 * n_masses, vel_out=3 * n_masses)
    for name, t in named.items():
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"titan_step_atomic_noalloc: {name} must be a torch tensor on {device}, "
                            f"not {type(t).__name__}")
        if t.device != device:
            raise ValueError(f"titan_step_atomic_noalloc: {name} is on {t.device}, expected {device}")
        want = (torch.int32,) if name == "ends" else (torch.float32,)
        if t.dtype not in want:
            raise TypeError(f"titan_step_atomic_noalloc: {name} has dtype {t.dtype}, expected {want[0]}")
        if not t.is_contiguous():
            raise ValueError(f"titan_step_atomic_noalloc: {name} must be contiguous")
        if t.numel() != sizes[name]:
            raise ValueError(f"titan_step_atomic_noalloc: {name} has {t.numel()} elements, expected {sizes[name]}")

    def span(t):
        a = t.data_ptr()
        return a, a + t.numel() * t.element_size()

    for out in ("pos_out", "vel_out"):
        o0, o1 = span(named[out])
        for name, t in named.items():
            if name == out or t.numel() == 0 or named[out].numel() == 0:
                continue
            a0, a1 = span(t)
            if o0 < a1 and a0 < o1:
                raise ValueError(f"titan_step_atomic_noalloc: {out} overlaps {name}")


def titan_step_atomic_noalloc(n_masses: int, pos_dev, vel_dev, inv_mass_dev, n_springs: int, ends_dev,
                              k_dev, rest_dev, damping: float, params: titan_params, pos_out_dev,
                              vel_out_dev, stream: Optional[int] = None) -> None:
    """One atomic-scatter step on caller-owned device tensors, allocating
    nothing (the accumulator is a fixed array inside the library).  The
    tensors are checked first (check_noalloc_args): float32 (ends int32),
    contiguous, on the current CUDA device, of the sizes the counts imply,
    outputs apart from every input."""
    check_noalloc_args(n_masses, n_springs, pos_dev, vel_dev, inv_mass_dev, ends_dev, k_dev, rest_dev,
                       pos_out_dev, vel_out_dev)
    _check(load().titan_step_atomic_noalloc(
        n_masses, _ptr(pos_dev), _ptr(vel_dev), _ptr(inv_mass_dev), n_springs, _ptr(ends_dev),
        _ptr(k_dev), _ptr(rest_dev), float(damping), C.byref(params), _ptr(pos_out_dev),
        _ptr(vel_out_dev), stream))


def titan_selftest_wait_timeout(device: int = 0, spin_limit: int = 4096) -> int:
    """Runs the bounded-wait failure self-test on `device` and returns its
    status: TITAN_E_TIMEOUT (4) is the expected outcome.  Other statuses
    raise TitanError."""
    st = load().titan_selftest_wait_timeout(device, spin_limit)
    if st != TITAN_E_TIMEOUT:
        _check(st)
        raise TitanError(st, "titan_selftest_wait_timeout: the wait did not expire")
    return st


def _bcheck(status: int, batch=None):
    if status != TITAN_OK:
        lib = load()
        msg = (lib.titan_batch_last_error(batch) if batch else lib.titan_last_error(None))
        raise TitanError(status, msg.decode(errors="replace"))


def _params_from(system, device=0, stream=None):
    p = titan_default_params()
    p.dt = float(system.dt)
    p.gravity = (C.c_double * 3)(*[float(g) for g in system.gravity])
    p.ground = 1 if system.ground else 0
    p.ground_k = float(system.ground_k)
    p.mu = float(system.mu)
    p.device = device
    p.stream = stream
    return p


class Batch:
    """Many independent systems advanced together (titan_batch_* calls).

    All systems share dt, gravity, ground parameters and one uniform damping
    (taken from the first system) and one actuation frequency."""

    def __init__(self, systems, device: int = 0, stream: Optional[int] = None):
        load()
        self.n = len(systems)
        self.sizes = [int(sy.pos.shape[0]) for sy in systems]
        keep, ms, ss, acts = [], [], [], []
        damping = float(systems[0].damping[0]) if systems and len(systems[0].damping) else 0.0
        for sy in systems:
            d = dict(pos=np.ascontiguousarray(sy.pos, np.float64), vel=np.ascontiguousarray(sy.vel, np.float64),
                     mass=np.ascontiguousarray(sy.mass, np.float64),
                     fixed=np.ascontiguousarray(sy.fixed, np.uint8),
                     ends=np.ascontiguousarray(sy.ends, np.uint32), k=np.ascontiguousarray(sy.k, np.float64),
                     rest=np.ascontiguousarray(sy.rest, np.float64))
            if len(sy.damping) and not np.all(sy.damping == damping):
                raise ValueError("a batch uses one uniform damping")
            ms.append(titan_masses(sy.n_masses, _ptr(d["pos"]), _ptr(d["vel"]), _ptr(d["mass"]), _ptr(d["fixed"])))
            ss.append(titan_springs(sy.n_springs, _ptr(d["ends"]), _ptr(d["k"]), _ptr(d["rest"]), None))
            if getattr(sy, "act_amp", None) is not None:
                d["amp"] = np.ascontiguousarray(sy.act_amp, np.float64)
                d["phase"] = np.ascontiguousarray(sy.act_phase, np.float64)
                acts.append(titan_actuation(_ptr(d["amp"]), _ptr(d["phase"]), float(sy.act_freq)))
            else:
                acts.append(titan_actuation(None, None, 0.0))
            keep.append(d)
        p = _params_from(systems[0], device, stream)
        p.damping = damping
        M = (titan_masses * max(1, self.n))(*ms)
        S = (titan_springs * max(1, self.n))(*ss)
        A = (titan_actuation * max(1, self.n))(*acts)
        out = _P()
        _bcheck(load().titan_batch_create(self.n, M, S, A, C.byref(p), C.byref(out)))
        self.handle = out.value

    def rollout(self, n_steps: int) -> "Batch":
        _bcheck(load().titan_batch_rollout(self.handle, n_steps), self.handle)
        return self

    def autotune(self, probe_steps: int = 50) -> None:
        _bcheck(load().titan_batch_autotune(self.handle, probe_steps), self.handle)

    def reset(self) -> None:
        _bcheck(load().titan_batch_reset(self.handle), self.handle)

    def sync(self) -> None:
        _bcheck(load().titan_batch_sync(self.handle), self.handle)

    def group_of(self, r: int) -> int:
        """Index (into groups()) of the launch group that advances system r."""
        g = C.c_uint32()
        _bcheck(load().titan_batch_system_group(self.handle, r, C.byref(g)), self.handle)
        return int(g.value)

    def read(self, r: int):
        n = self.sizes[r]
        pos = np.empty((n, 3), np.float32)
        vel = np.empty((n, 3), np.float32)
        _bcheck(load().titan_batch_read(self.handle, r, _ptr(pos), _ptr(vel)), self.handle)
        return pos, vel

    def centroids(self) -> np.ndarray:
        out = np.empty((self.n, 3), np.float32)
        _bcheck(load().titan_batch_centroids(self.handle, _ptr(out)), self.handle)
        return out

    def configure(self, group: int, threads: int, threads_per_mass: int) -> None:
        _bcheck(load().titan_batch_configure(self.handle, group, threads, threads_per_mass), self.handle)

    def groups(self):
        lib = load()
        res = []
        for g in range(lib.titan_batch_groups(self.handle)):
            cl, th, tm, ct = C.c_uint32(), C.c_uint32(), C.c_uint32(), C.c_uint32()
            _bcheck(lib.titan_batch_info(self.handle, g, C.byref(cl), C.byref(th), C.byref(tm), C.byref(ct)),
                    self.handle)
            res.append(dict(cluster=cl.value, threads=th.value, threads_per_mass=tm.value, ctas=ct.value))
        return res

    def close(self) -> None:
        if getattr(self, "handle", None):
            _bcheck(load().titan_batch_destroy(self.handle))
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------------- convenience

class Sim:
    """Owns one titan_sim handle built from an ``inputs.System``-like object."""

    def __init__(self, system, accumulate: int = ACCUM_CSR, order: int = ORDER_MORTON,
                 exec_mode: int = EXEC_AUTO, graph_chunk: int = 0, stream: Optional[int] = None,
                 device: int = 0, kernel_variant: int = 0, l2_persist: bool = True, launch_overlap: bool = True):
        load()
        self.n = int(system.pos.shape[0])
        self.s = int(system.ends.shape[0])
        self.dt = float(system.dt)
        self._keep = dict(
            pos=np.ascontiguousarray(system.pos, dtype=np.float64),
            vel=np.ascontiguousarray(system.vel, dtype=np.float64),
            mass=np.ascontiguousarray(system.mass, dtype=np.float64),
            fixed=np.ascontiguousarray(system.fixed, dtype=np.uint8),
            ends=np.ascontiguousarray(system.ends, dtype=np.uint32),
            k=np.ascontiguousarray(system.k, dtype=np.float64),
            # rest None: NULL, the library takes each spring's initial length
            rest=None if system.rest is None else np.ascontiguousarray(system.rest, dtype=np.float64),
            damping=np.ascontiguousarray(system.damping, dtype=np.float64))
        kp = self._keep
        m = titan_masses(self.n, _ptr(kp["pos"]), _ptr(kp["vel"]), _ptr(kp["mass"]), _ptr(kp["fixed"]))
        sp = titan_springs(self.s, _ptr(kp["ends"]), _ptr(kp["k"]), _ptr(kp["rest"]), _ptr(kp["damping"]))
        p = titan_default_params()
        p.dt = self.dt
        p.gravity = (C.c_double * 3)(*[float(g) for g in system.gravity])
        p.ground = 1 if system.ground else 0
        p.ground_k = float(system.ground_k)
        p.mu = float(system.mu)
        p.accumulate, p.order, p.exec, p.device = accumulate, order, exec_mode, device
        p.graph_chunk = graph_chunk
        p.kernel_variant = kernel_variant
        p.l2_persist = 1 if l2_persist else 0
        p.launch_overlap = 1 if launch_overlap else 0
        p.stream = stream
        self.handle = titan_create(m, sp, p)
        self._keep = None
        if getattr(system, "act_amp", None) is not None:
            ids = np.arange(self.s, dtype=np.uint32)
            titan_set_actuation(self.handle, ids, system.act_amp, system.act_phase, system.act_freq)

    def step(self, n: int) -> "Sim":
        titan_step(self.handle, n)
        return self

    def snapshot(self, copy: bool = True):
        """(pos, vel, t) after every step enqueued so far (float32, caller order);
        copy=False: read-only views of the pinned snapshot buffers, valid until
        the second next snapshot."""
        t = titan_snapshot_async(self.handle)          # first: a pending rebuild changes n
        return titan_snapshot_wait(self.handle, t, self.n, copy=copy)

    def add_masses(self, pos, mass, vel=None, fixed=None) -> int:
        first = titan_add_masses(self.handle, pos, mass, vel, fixed)
        self.n += int(np.asarray(mass).size)
        return first

    def add_springs(self, ends, k, rest=None, damping=None) -> int:
        first = titan_add_springs(self.handle, ends, k, rest, damping)
        self.s += int(np.asarray(ends).size // 2)
        return first

    def set_state(self, pos, vel=None) -> None:
        titan_set_state(self.handle, pos, vel)

    def sync(self) -> None:
        titan_sync(self.handle)

    @property
    def steps(self) -> int:
        return titan_steps(self.handle)

    @property
    def exec_mode(self) -> int:
        """EXEC_PERSISTENT or EXEC_LAUNCH: how titan_step runs this system."""
        return int(load().titan_exec_mode(self.handle))

    @property
    def csr_kernel(self) -> int:
        """The step kernel in use: 1..9 (see titan_params.kernel_variant), 0 atomic."""
        return int(load().titan_csr_kernel(self.handle))

    def close(self) -> None:
        if getattr(self, "handle", None):
            titan_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------------- differentiable rollouts

def union_system(systems):
    """Concatenates independent systems into one (block-diagonal) system.
    Returns (system, mass_offsets, spring_offsets)."""
    from .inputs import System
    mo = np.cumsum([0] + [sy.n_masses for sy in systems])
    so = np.cumsum([0] + [sy.n_springs for sy in systems])
    cat = lambda f: np.concatenate([getattr(sy, f) for sy in systems])
    ends = np.concatenate([sy.ends.astype(np.int64) + mo[r] for r, sy in enumerate(systems)]).astype(np.uint32)
    s0 = systems[0]
    amp = np.concatenate([sy.act_amp if sy.act_amp is not None else np.zeros(sy.n_springs) for sy in systems])
    ph = np.concatenate([sy.act_phase if sy.act_phase is not None else np.zeros(sy.n_springs) for sy in systems])
    u = System(pos=cat("pos"), vel=cat("vel"), mass=cat("mass"), fixed=cat("fixed"), ends=ends, k=cat("k"),
               rest=cat("rest"), damping=cat("damping"), dt=s0.dt, gravity=s0.gravity, ground=s0.ground,
               ground_k=s0.ground_k, mu=s0.mu, act_amp=amp, act_phase=ph, act_freq=s0.act_freq,
               spacing=s0.spacing, name="union")
    return u, mo, so


class CentroidRollout:
    """Centroid x-displacement of each of several robots after an n_steps
    rollout, as a differentiable function of every spring's actuation
    amplitude and phase (concatenated over the robots, robot by robot).

    ``__call__(amp, phase)`` takes CUDA float32 tensors and returns a tensor
    of per-robot displacements; gradients flow back through the library's
    adjoint (titan_adjoint) with checkpoints every ``every`` steps."""

    def __init__(self, robots, n_steps: int, every: int = 50, device: int = 0, order: int = ORDER_MORTON):
        import torch
        self.system, self.mass_off, self.spring_off = union_system(robots)
        self.n_steps, self.every = int(n_steps), int(every)
        self.n_robots = len(robots)
        self.freq = float(self.system.act_freq)
        self.device = device
        self.sim = Sim(self.system, device=device, order=order)
        self.pos0 = np.ascontiguousarray(self.system.pos)
        self.vel0 = np.ascontiguousarray(self.system.vel)
        self.x0 = np.array([self.pos0[self.mass_off[r]:self.mass_off[r + 1], 0].mean()
                            for r in range(self.n_robots)])
        self._fn = None
        self._dev = None
        self._torch = torch

    def _dev_tables(self):
        """The robots' mass ranges (uint32 offsets) and initial centroids
        (float32 [robots][3]), kept on the device after the first use."""
        if self._dev is None:
            T_ = self._torch
            dev = T_.device("cuda", self.device)
            first = T_.as_tensor(np.asarray(self.mass_off, np.int64).astype(np.int32), device=dev)
            origin = np.zeros((self.n_robots, 3), np.float32)
            origin[:, 0] = self.x0
            self._dev = (first, T_.as_tensor(origin, device=dev))
        return self._dev

    def _prepare(self, amp, phase):
        T_ = self._torch
        dev = T_.device("cuda", self.device)
        a = amp.detach().to(dev, T_.float32).contiguous()
        p = phase.detach().to(dev, T_.float32).contiguous()
        T_.cuda.current_stream(dev).synchronize()      # the library reads them on its own stream
        titan_set_actuation_dev(self.sim.handle, a, p, self.freq)
        titan_set_step(self.sim.handle, 0)
        self.sim.set_state(self.pos0, self.vel0)

    def forward(self, amp, phase):
        T_ = self._torch
        self._prepare(amp, phase)
        self.sim.step(self.n_steps)
        first, origin = self._dev_tables()
        out = T_.empty((self.n_robots, 3), dtype=T_.float32, device=f"cuda:{self.device}")
        titan_group_centroids(self.sim.handle, first, origin, out)     # displacement of every centroid
        self.sim.sync()
        return out[:, 0].contiguous()

    def gradients(self, amp, phase, grad_out):
        """dJ/dA and dJ/dphi for the objective sum_r grad_out[r] * J_r."""
        T_ = self._torch
        self._prepare(amp, phase)
        dev = f"cuda:{self.device}"
        first, _ = self._dev_tables()
        w = grad_out.detach().to(dev, T_.float32).contiguous()
        seed = T_.empty((self.system.n_masses, 3), dtype=T_.float32, device=dev)
        ga = T_.empty(self.system.n_springs, dtype=T_.float32, device=dev)
        gp = T_.empty_like(ga)
        T_.cuda.current_stream(dev).synchronize()      # w is written on torch's stream
        titan_group_seed(self.sim.handle, first, w, 0, seed)
        titan_adjoint(self.sim.handle, self.n_steps, self.every, seed, None, ga, gp)
        self.sim.sync()
        return ga, gp

    def __call__(self, amp, phase):
        if self._fn is None:
            torch = self._torch
            engine = self

            class _Fn(torch.autograd.Function):
                @staticmethod
                def forward(ctx, a, p):
                    ctx.save_for_backward(a, p)
                    return engine.forward(a, p)

                @staticmethod
                def backward(ctx, g):
                    a, p = ctx.saved_tensors
                    ga, gp = engine.gradients(a, p, g)
                    return ga.to(a.dtype), gp.to(p.dtype)

            self._fn = _Fn
        return self._fn.apply(amp, phase)


# --------------------------------------------------------------------------- tensor-core surrogate MLP

def titan_gemm_bf16_tn(A, B, C, stream: Optional[int] = None) -> None:
    """C = A B^T on the tcgen05 tensor cores (A, B: CUDA bfloat16 tensors [M, K], [N, K]; C: float32 [M, N]),
    enqueued on `stream` (default: torch's current stream of A's device); returns without waiting."""
    M, K = A.shape
    N = B.shape[0]
    if stream is None:
        import torch
        stream = torch.cuda.current_stream(A.device).cuda_stream
    _check_mlp(load().titan_gemm_bf16_tn(M, N, K, _ptr(A), _ptr(B), _ptr(C), stream))


def titan_gemm_check() -> None:
    """Raises TitanError (TITAN_E_TIMEOUT) if a GEMM kernel on the current
    device gave up on a bounded wait since the last check."""
    _check_mlp(load().titan_gemm_check())


def _check_mlp(status: int, m=None):
    if status != TITAN_OK:
        lib = load()
        msg = lib.titan_mlp_last_error(m) if m else lib.titan_last_error(None)
        raise TitanError(status, msg.decode(errors="replace"))


class MLP:
    """The surrogate network (titan_mlp_*): in -> hidden x 3 (GELU) -> 1."""

    def __init__(self, n_in: int = 1024, hidden: int = 512, seed: int = 0, device: int = 0,
                 stream: Optional[int] = None):
        load()
        out = _P()
        _check_mlp(load().titan_mlp_create(n_in, hidden, seed, device, stream, C.byref(out)))
        self.handle = out.value
        self.n_in, self.hidden = n_in, hidden
        self.n_params = int(load().titan_mlp_param_count(self.handle))

    def get_params(self) -> np.ndarray:
        p = np.empty(self.n_params, np.float32)
        _check_mlp(load().titan_mlp_get_params(self.handle, _ptr(p)), self.handle)
        return p

    def set_params(self, p) -> None:
        p = np.ascontiguousarray(p, np.float32)
        _check_mlp(load().titan_mlp_set_params(self.handle, _ptr(p)), self.handle)

    def forward(self, x, y) -> None:
        _check_mlp(load().titan_mlp_forward(self.handle, _ptr(x), x.shape[0], _ptr(y)), self.handle)

    def gradient(self, x, t, loss, grad) -> None:
        _check_mlp(load().titan_mlp_gradient(self.handle, _ptr(x), _ptr(t), x.shape[0], _ptr(loss), _ptr(grad)),
                   self.handle)

    def train_step(self, x, t, lr: float, loss=None) -> None:
        _check_mlp(load().titan_mlp_train_step(self.handle, _ptr(x), _ptr(t), x.shape[0], float(lr), _ptr(loss)),
                   self.handle)

    def sync(self) -> None:
        _check_mlp(load().titan_mlp_sync(self.handle), self.handle)

    def unpack(self, p):
        """Splits a flat parameter vector into (W1t, b1, W2t, b2, W3t, b3, w4, b4)."""
        h, i = self.hidden, self.n_in
        out, o = [], 0
        for shape in [(h, i), (h,), (h, h), (h,), (h, h), (h,), (h,), (1,)]:
            n = int(np.prod(shape))
            out.append(np.asarray(p[o:o + n]).reshape(shape))
            o += n
        return out

    def close(self) -> None:
        if getattr(self, "handle", None):
            load().titan_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

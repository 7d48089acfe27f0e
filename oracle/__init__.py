"""ctypes wrapper around the FP64 CPU oracle (titan_oracle.c).

TEST INFRASTRUCTURE ONLY: only tests/, the smoke check and the benchmark's
CPU-baseline leg may import this package.  The product path (the CUDA library
and its Python binding) never imports it.

``build()`` compiles titan_oracle.c with gcc into oracle/_build/liboracle.so;
``run()`` advances a copy of a system's state; ``spring_forces()`` evaluates the
spring pass alone.  Arrays are passed as FP64 (and uint32/uint8) numpy arrays.
"""
from __future__ import annotations

import contextlib
import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "titan_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_SRC_OMP = os.path.join(_HERE, "titan_oracle_omp.c")
_LIB_OMP_PATH = os.path.join(_OUT_DIR, "liboracle_omp.so")
_lib = None
_lib_omp = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                           "-fno-fast-math", _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def build_parallel(force: bool = False) -> str:
    """Compile the all-cores variant (titan_oracle_omp.c, OpenMP) into
    oracle/_build/liboracle_omp.so, with the serial oracle's flags."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_OMP))
    if not force and os.path.exists(_LIB_OMP_PATH) and os.path.getmtime(_LIB_OMP_PATH) >= newest:
        return _LIB_OMP_PATH
    tmp = _LIB_OMP_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                           "-fno-fast-math", "-fopenmp", "-I", _HERE, _SRC_OMP, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB_OMP_PATH)
    return _LIB_OMP_PATH


class OracleSystem(C.Structure):
    _fields_ = [
        ("n_masses", C.c_int64), ("n_springs", C.c_int64),
        ("mass", C.c_void_p), ("fixed", C.c_void_p), ("ends", C.c_void_p),
        ("k", C.c_void_p), ("rest", C.c_void_p), ("damping", C.c_void_p),
        ("act_a", C.c_void_p), ("act_b", C.c_void_p),
        ("act_mode", C.c_int32), ("ground", C.c_int32),
        ("act_freq", C.c_double), ("worm_omega", C.c_double), ("worm_period", C.c_double),
        ("dt", C.c_double), ("gravity", C.c_double * 3),
        ("ground_k", C.c_double), ("mu", C.c_double),
    ]


def _bind(lib):
    P = C.POINTER(OracleSystem)
    lib.titan_oracle_run.argtypes = [P, C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_void_p]
    lib.titan_oracle_run.restype = None
    lib.titan_oracle_spring_forces.argtypes = [P, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]
    lib.titan_oracle_spring_forces.restype = None
    lib.titan_oracle_mass_update.argtypes = [P, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.titan_oracle_mass_update.restype = None
    lib.titan_oracle_rest_length.argtypes = [P, C.c_int64, C.c_double]
    lib.titan_oracle_rest_length.restype = C.c_double
    lib.titan_oracle_adjoint.argtypes = [P, C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_void_p,
                                         C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.titan_oracle_adjoint.restype = C.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(C.CDLL(build()))
    return _lib


def _load_parallel():
    global _lib_omp
    with _lock:
        if _lib_omp is None:
            lib = C.CDLL(build_parallel())
            P = C.POINTER(OracleSystem)
            lib.titan_oracle_incidence.argtypes = [P, C.c_void_p, C.c_void_p]
            lib.titan_oracle_incidence.restype = None
            lib.titan_oracle_run_parallel.argtypes = [P, C.c_void_p, C.c_void_p, C.c_int64, C.c_int64,
                                                      C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
            lib.titan_oracle_run_parallel.restype = C.c_int
            lib.titan_oracle_max_threads.argtypes = []
            lib.titan_oracle_max_threads.restype = C.c_int
            _lib_omp = lib
    return _lib_omp


@contextlib.contextmanager
def mutant(source: str, workdir: str):
    """Temporarily replace the oracle with a build of ``source`` (a modified
    copy of titan_oracle.c).  Used only by the test that checks that the pins
    catch planted mistakes."""
    global _lib
    src = os.path.join(workdir, "mutant.c")
    out = os.path.join(workdir, f"libmutant{abs(hash(source))}.so")
    with open(src, "w") as f:
        f.write(source)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                           src, "-o", out, "-lm"])
    saved = _load()
    with _lock:
        _lib = _bind(C.CDLL(out))
    try:
        yield
    finally:
        with _lock:
            _lib = saved


def source() -> str:
    with open(_SRC) as f:
        return f.read()


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class _Bound:
    """Keeps the numpy arrays alive while the C struct points into them."""

    def __init__(self, sys, act_mode=None, worm=None):
        self.arrays = dict(
            mass=_f64(sys.mass), fixed=np.ascontiguousarray(sys.fixed, dtype=np.uint8),
            ends=np.ascontiguousarray(sys.ends, dtype=np.uint32), k=_f64(sys.k),
            rest=_f64(sys.rest), damping=_f64(sys.damping))
        st = OracleSystem()
        st.n_masses = sys.n_masses
        st.n_springs = sys.n_springs
        for name in ("mass", "fixed", "ends", "k", "rest", "damping"):
            setattr(st, name, self.arrays[name].ctypes.data)
        mode = act_mode if act_mode is not None else (1 if sys.act_amp is not None else 0)
        st.act_mode = mode
        if mode:
            self.arrays["act_a"] = _f64(sys.act_amp)
            self.arrays["act_b"] = _f64(sys.act_phase)
            st.act_a = self.arrays["act_a"].ctypes.data
            st.act_b = self.arrays["act_b"].ctypes.data
        st.act_freq = float(sys.act_freq)
        if worm is not None:
            st.worm_omega, st.worm_period = float(worm[0]), float(worm[1])
        st.ground = 1 if sys.ground else 0
        st.dt = float(sys.dt)
        st.gravity = (C.c_double * 3)(*[float(g) for g in sys.gravity])
        st.ground_k = float(sys.ground_k)
        st.mu = float(sys.mu)
        self.struct = st


def run(sys, n_steps: int, step0: int = 0, pos=None, vel=None, act_mode=None, worm=None):
    """Advance (pos, vel) (default: the system's own) by n_steps; returns copies."""
    lib = _load()
    b = _Bound(sys, act_mode, worm)
    x = _f64(sys.pos if pos is None else pos).copy()
    v = _f64(sys.vel if vel is None else vel).copy()
    F = np.empty_like(x)
    lib.titan_oracle_run(C.byref(b.struct), x.ctypes.data, v.ctypes.data, int(step0), int(n_steps),
                         F.ctypes.data)
    return x, v


class Parallel:
    """The all-cores variant bound to one system: its per-mass incidence is
    built once; run() then advances a state like the serial run() (the same
    trajectory, bit for bit) on `threads` threads (0: all cores)."""

    def __init__(self, sys, act_mode=None, worm=None, threads: int = 0):
        self.lib = _load_parallel()
        self.sys = sys
        self.bound = _Bound(sys, act_mode, worm)
        self.rowptr = np.zeros(sys.n_masses + 1, np.int64)
        self.ent = np.zeros(max(1, 2 * sys.n_springs), np.uint64)
        self.lib.titan_oracle_incidence(C.byref(self.bound.struct), self.rowptr.ctypes.data, self.ent.ctypes.data)
        self.threads = int(threads)
        self.threads_used = 0

    def run(self, n_steps: int, step0: int = 0, pos=None, vel=None):
        x = _f64(self.sys.pos if pos is None else pos).copy()
        v = _f64(self.sys.vel if vel is None else vel).copy()
        F = np.empty_like(x)
        self.threads_used = self.lib.titan_oracle_run_parallel(
            C.byref(self.bound.struct), x.ctypes.data, v.ctypes.data, int(step0), int(n_steps), F.ctypes.data,
            self.rowptr.ctypes.data, self.ent.ctypes.data, self.threads)
        return x, v


def run_parallel(sys, n_steps: int, step0: int = 0, pos=None, vel=None, act_mode=None, worm=None,
                 threads: int = 0):
    """run() on all cores (or `threads`): the same trajectory, bit for bit."""
    return Parallel(sys, act_mode, worm, threads).run(n_steps, step0, pos, vel)


def max_threads() -> int:
    return int(_load_parallel().titan_oracle_max_threads())


def spring_forces(sys, pos=None, vel=None, step: int = 0, act_mode=None, worm=None):
    """The spring pass alone: the (n, 3) force each mass receives from springs."""
    lib = _load()
    b = _Bound(sys, act_mode, worm)
    x = _f64(sys.pos if pos is None else pos)
    v = _f64(sys.vel if vel is None else vel)
    F = np.empty_like(x)
    lib.titan_oracle_spring_forces(C.byref(b.struct), x.ctypes.data, v.ctypes.data, int(step),
                                   F.ctypes.data)
    return F


def rest_length(sys, s: int, t: float, act_mode=None, worm=None) -> float:
    lib = _load()
    b = _Bound(sys, act_mode, worm)
    return lib.titan_oracle_rest_length(C.byref(b.struct), int(s), float(t))


def adjoint(sys, n_steps: int, seed_x, seed_v=None, step0: int = 0, pos=None, vel=None):
    """Reverse-mode gradient of J = <seed_x, x_T> + <seed_v, v_T> with respect
    to the actuation amplitudes and phases of every spring.
    Returns (grad_amp, grad_phase, x_T, v_T)."""
    lib = _load()
    b = _Bound(sys, 1, None)
    x0 = _f64(sys.pos if pos is None else pos)
    v0 = _f64(sys.vel if vel is None else vel)
    sx = _f64(seed_x)
    sv = None if seed_v is None else _f64(seed_v)
    ga = np.zeros(sys.n_springs)
    gb = np.zeros(sys.n_springs)
    xT = np.empty_like(x0)
    vT = np.empty_like(v0)
    rc = lib.titan_oracle_adjoint(C.byref(b.struct), x0.ctypes.data, v0.ctypes.data, int(step0), int(n_steps),
                                  sx.ctypes.data, None if sv is None else sv.ctypes.data,
                                  ga.ctypes.data, gb.ctypes.data, xT.ctypes.data, vT.ctypes.data)
    if rc != 0:
        raise RuntimeError("oracle adjoint failed (needs sinusoidal actuation)")
    return ga, gb, xT, vT


def centroid_x_seed(n: int) -> np.ndarray:
    """Seed for J = mean_i x_T[i, 0] (the centroid's x position)."""
    s = np.zeros((n, 3))
    s[:, 0] = 1.0 / n
    return s

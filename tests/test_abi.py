"""The C-ABI library: it builds, loads, exports every declared symbol, and
validates its inputs on the host before touching a GPU (these run on CPU)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1911_10274_gb300 import inputs
from paper_1911_10274_gb300 import titan as T

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[\w\s\*]*?\b(titan_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("titan_create", "titan_step", "titan_snapshot_async", "titan_snapshot_wait",
                     "titan_set_actuation", "titan_destroy", "titan_sync", "titan_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = T.load()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_library_links_only_the_cuda_runtime_not_torch():
    import subprocess
    out = subprocess.run(["ldd", T._build.LIB_PATH], capture_output=True, text=True).stdout
    assert "libcudart" in out
    assert "torch" not in out and "python" not in out


def test_default_params():
    p = T.titan_default_params()
    assert p.dt == 1e-4 and list(p.gravity) == [0.0, 0.0, -9.81]
    assert p.accumulate == T.ACCUM_CSR and p.order == T.ORDER_MORTON and p.exec == T.EXEC_AUTO
    assert p.l2_persist == 1 and p.launch_overlap == 1 and list(p.reserved) == [0] * 4


def test_binding_structs_match_the_header(tmp_path):
    """The ctypes mirrors of the ABI structs have the header's sizes and offsets."""
    import ctypes
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    src = tmp_path / "sz.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "titan.h"\n'
                   'int main(void) { printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(titan_params), '
                   'offsetof(titan_params, stream), offsetof(titan_params, kernel_variant), '
                   'offsetof(titan_params, l2_persist), sizeof(titan_masses), sizeof(titan_springs)); return 0; }\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [ctypes.sizeof(T.titan_params), T.titan_params.stream.offset, T.titan_params.kernel_variant.offset,
            T.titan_params.l2_persist.offset, ctypes.sizeof(T.titan_masses), ctypes.sizeof(T.titan_springs)]
    assert got == want


def _arrays(sys):
    keep = dict(pos=np.ascontiguousarray(sys.pos), mass=np.ascontiguousarray(sys.mass),
                ends=np.ascontiguousarray(sys.ends, np.uint32), k=np.ascontiguousarray(sys.k),
                rest=np.ascontiguousarray(sys.rest), damping=np.ascontiguousarray(sys.damping))
    m = T.titan_masses(sys.n_masses, keep["pos"].ctypes.data, None, keep["mass"].ctypes.data, None)
    s = T.titan_springs(sys.n_springs, keep["ends"].ctypes.data, keep["k"].ctypes.data,
                        keep["rest"].ctypes.data, keep["damping"].ctypes.data)
    return keep, m, s


@pytest.mark.parametrize("mutate,needle", [
    (lambda d: d["ends"].__setitem__((0, 1), 99), "out of range"),
    (lambda d: d["ends"].__setitem__((0, 1), d["ends"][0, 0]), "itself"),
    (lambda d: d["k"].__setitem__(3, -1.0), "springs.k"),
    (lambda d: d["k"].__setitem__(3, np.nan), "springs.k"),
    (lambda d: d["rest"].__setitem__(2, np.inf), "springs.rest"),
    (lambda d: d["damping"].__setitem__(2, -0.5), "springs.damping"),
    (lambda d: d["mass"].__setitem__(1, 0.0), "masses.mass"),
    (lambda d: d["pos"].__setitem__((1, 2), np.nan), "masses.pos"),
])
def test_create_rejects_invalid_inputs_before_touching_the_device(mutate, needle):
    sys = inputs.cube_drop(n=2)
    keep, m, s = _arrays(sys)
    mutate(keep)
    with pytest.raises(T.TitanError) as ei:
        T.titan_create(m, s, T.titan_default_params())
    assert ei.value.status == T.TITAN_E_INVALID
    assert needle in str(ei.value)


@pytest.mark.parametrize("field,value", [("dt", 0.0), ("dt", float("nan")), ("mu", -1.0),
                                         ("ground_k", float("inf")), ("accumulate", 7),
                                         ("order", 3), ("exec", 9), ("device", -1)])
def test_create_rejects_invalid_params(field, value):
    sys = inputs.cube_drop(n=2)
    keep, m, s = _arrays(sys)
    p = T.titan_default_params()
    setattr(p, field, value)
    with pytest.raises(T.TitanError) as ei:
        T.titan_create(m, s, p)
    assert ei.value.status == T.TITAN_E_INVALID


def test_null_handle_calls_are_rejected():
    lib = T.load()
    assert lib.titan_step(None, 1) == T.TITAN_E_INVALID
    assert lib.titan_sync(None) == T.TITAN_E_INVALID
    assert lib.titan_destroy(None) == T.TITAN_OK
    assert lib.titan_steps(None) == 0
    assert isinstance(T.titan_last_error(None), str)


def test_batch_create_validates_before_touching_the_device():
    sy = inputs.actuated_box(3, 3, 3, np.random.default_rng(0))
    bad = sy.copy()
    bad.ends = bad.ends.copy()
    bad.ends[0, 1] = 500
    with pytest.raises(T.TitanError) as ei:
        T.Batch([sy, bad])
    assert ei.value.status == T.TITAN_E_INVALID and "system 1" in str(ei.value)
    other = sy.copy()
    other.act_freq = 3.0
    with pytest.raises(T.TitanError) as ei:
        T.Batch([sy, other])
    assert ei.value.status == T.TITAN_E_UNSUPPORTED


def test_wait_timeout_selftest_rejects_unbounded_limits_before_touching_the_device():
    for bad in (0, (1 << 20) + 1):
        with pytest.raises(T.TitanError, match="spin_limit"):
            T.titan_selftest_wait_timeout(0, bad)


def test_every_source_and_header_is_a_rebuild_input():
    """Editing any file of the kernel sources or the public header must make
    the library stale, headers of device code (.cuh) included."""
    from paper_1911_10274_gb300 import build as B
    watched = {os.path.abspath(f) for f in B._inputs()}
    for d in (B.CSRC, B.INCLUDE):
        for f in os.listdir(d):
            if f.endswith((".cu", ".cpp", ".h", ".cuh")):
                assert os.path.abspath(os.path.join(d, f)) in watched, f

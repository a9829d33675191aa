"""The C-ABI library loads and exports every function include/mdk.h declares
(no GPU needed: nothing here calls into CUDA)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
           if f.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(mdk_[a-z_0-9]+)\s*\(",
                             src, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2511_22951_gb300 import _build
    _build.build()
    return ctypes.CDLL(_build.LIB)


def test_header_declares_the_path():
    names = declared_functions()
    for must in ("mdk_create", "mdk_set_potential_lj", "mdk_set_potential_eam",
                 "mdk_build_neighbors", "mdk_compute", "mdk_step", "mdk_set_piston",
                 "mdk_set_window", "mdk_profiles"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_header():
    from paper_2511_22951_gb300 import mdk
    assert set(declared_functions()) <= set(mdk.SIGNATURES), \
        set(declared_functions()) - set(mdk.SIGNATURES)


def test_status_strings_without_gpu(lib):
    lib.mdk_status_string.restype = ctypes.c_char_p
    lib.mdk_status_string.argtypes = [ctypes.c_int]
    assert lib.mdk_status_string(0) == b"ok"
    assert b"overflow" in lib.mdk_status_string(-3)


def test_argument_checks_without_gpu(lib):
    """Host-side validation runs before any CUDA call."""
    import numpy as np
    P = ctypes.c_void_p
    h = P()
    lo = np.zeros(3)
    hi = np.full(3, 10.0)
    per = np.ones(3, dtype=np.int32)
    m = np.full(4, 39.948)
    f = lib.mdk_create
    f.argtypes = [ctypes.POINTER(P), P, P, P, ctypes.c_int64, P, ctypes.c_int, P]
    assert f(ctypes.byref(h), lo.ctypes.data, hi.ctypes.data, per.ctypes.data, 4,
             m.ctypes.data, 7, None) == -1          # bad precision
    assert f(ctypes.byref(h), lo.ctypes.data, hi.ctypes.data, per.ctypes.data, 4,
             m.ctypes.data, 0, None) == 0
    lib.mdk_set_potential_lj.argtypes = [P, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_int]
    assert lib.mdk_set_potential_lj(h, 0.0104, 3.405, 8.5125, 1) == 0
    lib.mdk_plan_neighbors.argtypes = [P, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                       ctypes.c_int]
    # periodic box of 10 Angstrom is shorter than rc + skin = 8.8125? no: allowed
    assert lib.mdk_plan_neighbors(h, 8.5125, 0.3, 0, 0) == 0
    assert lib.mdk_plan_neighbors(h, 9.9, 0.3, 0, 0) == -2   # box too small
    sz = ctypes.c_size_t()
    lib.mdk_workspace_size.argtypes = [P, ctypes.POINTER(ctypes.c_size_t)]
    assert lib.mdk_plan_neighbors(h, 8.5125, 0.3, 0, 0) == 0
    assert lib.mdk_workspace_size(h, ctypes.byref(sz)) == 0 and sz.value > 0
    # two-level lists: the outer skin must exceed the skin, and the cells of
    # rc + skin_outer must fit the periodic box; the workspace grows by the outer list
    lib.mdk_set_outer_skin.argtypes = [P, ctypes.c_double]
    one_level = sz.value
    assert lib.mdk_set_outer_skin(h, 0.2) == -1
    assert lib.mdk_set_outer_skin(h, -1.0) == -1
    assert lib.mdk_set_outer_skin(h, 1.2) == 0           # rc + 1.2 = 9.71 <= 10
    assert lib.mdk_workspace_size(h, ctypes.byref(sz)) == 0 and sz.value > one_level
    two_level = sz.value
    assert lib.mdk_set_outer_skin(h, 2.0) == -2          # rc + 2.0 > 10: box too small
    assert lib.mdk_workspace_size(h, ctypes.byref(sz)) == 0 and sz.value == two_level
    assert lib.mdk_set_outer_skin(h, 0.0) == 0
    assert lib.mdk_workspace_size(h, ctypes.byref(sz)) == 0 and sz.value == one_level
    lib.mdk_step.argtypes = [P, ctypes.c_double, ctypes.c_int64]
    assert lib.mdk_step(h, 1.0, 1) == -8                # no workspace yet
    lib.mdk_get_build_counts.argtypes = [P, ctypes.c_void_p, ctypes.c_void_p]
    assert lib.mdk_get_build_counts(h, None, None) == -8
    assert lib.mdk_get_build_counts(None, None, None) == -1
    lib.mdk_destroy.argtypes = [P]
    assert lib.mdk_destroy(h) == 0


def test_debug_build_compiles():
    """The kernels compile with their debug-build index checks (MDK_DEBUG)."""
    import shutil
    import subprocess
    import tempfile
    from paper_2511_22951_gb300 import _build
    if shutil.which(_build.nvcc()) is None and not os.path.exists(_build.nvcc()):
        pytest.skip("no nvcc")
    src = os.path.join(_build.CSRC, "k_build.cu")
    with tempfile.TemporaryDirectory() as d:
        cmd = [_build.nvcc(), *_build.ARCH, *_build.NVCC_FLAGS, *_build.DEBUG_FLAGS, "-I",
               _build.INCLUDE, "-I", _build.CSRC, "-c", src, "-o", os.path.join(d, "k.o")]
        r = subprocess.run(cmd, capture_output=True, text=True)
        assert r.returncode == 0, r.stderr

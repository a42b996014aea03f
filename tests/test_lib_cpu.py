"""Host-side checks of the C-ABI library that need no GPU: it loads, and it
exports every entry point include/tomo.h declares."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2003_12677_b300 import build
    return build.build()


def declared():
    src = open(os.path.join(ROOT, "include", "tomo.h")).read()
    return sorted(set(re.findall(r"TOMO_API\s+[\w\s\*]*?\b(tomo_\w+)\s*\(", src)))


def test_header_declares_entry_points():
    names = declared()
    for n in ("tomo_build_matrix", "tomo_project", "tomo_backproject", "tomo_sirt", "tomo_cgls"):
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in declared():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (tomo_\w+)", out))
    assert set(declared()) <= exported
    # nothing but the declared C entry points is exported with the tomo_ prefix
    assert exported <= set(declared())


def test_binding_lists_every_symbol():
    from paper_2003_12677_b300 import _lib
    assert sorted(_lib.EXPORTS) == declared()


def test_status_strings(lib_path):
    lib = ctypes.CDLL(lib_path)
    lib.tomo_status_string.restype = ctypes.c_char_p
    assert lib.tomo_status_string(0) == b"TOMO_OK"
    assert lib.tomo_status_string(4) == b"TOMO_ERR_TIMEOUT"


def test_invalid_arguments_rejected_without_gpu(lib_path):
    """Argument validation happens on the host before any CUDA call."""
    from paper_2003_12677_b300 import _lib
    lib = _lib.load(lib_path)
    g = _lib.Geometry()
    g.n_x, g.n_y, g.n_p, g.n_theta = 0, 4, 4, 4
    g.center = float("nan")
    h = ctypes.c_void_p()
    assert lib.tomo_build_matrix(ctypes.byref(g), None, None, ctypes.byref(h)) == 1
    assert b"positive" in lib.tomo_last_error()
    g.n_x = 4
    opts = _lib.MatrixOpts()
    opts.values = 9
    assert lib.tomo_build_matrix(ctypes.byref(g), ctypes.byref(opts), None, ctypes.byref(h)) == 1
    g.n_x, g.n_y = 70000, 70000
    assert lib.tomo_build_matrix(ctypes.byref(g), None, None, ctypes.byref(h)) == 1
    assert lib.tomo_project(None, None, None, 1, 0, None, None, 0, None) == 1
    assert lib.tomo_sirt(None, None, None, 1, 1, ctypes.c_float(1.0), None, None, 0, None) == 1


def test_more_arguments_rejected_without_gpu(lib_path):
    """TV's eps must have a normal FP32 square; the data-fit call needs its buffers."""
    import numpy as np
    from paper_2003_12677_b300 import _lib
    lib = _lib.load(lib_path)
    buf = np.zeros(64, np.float64)        # host memory, 16-byte aligned; never dereferenced here
    p = ctypes.c_void_p(buf.ctypes.data)
    assert buf.ctypes.data % 16 == 0
    assert lib.tomo_tv(p, 1, 2, 2, ctypes.c_float(1e-20), p, p, None) == 1
    assert b"eps" in lib.tomo_last_error()
    assert lib.tomo_residual_norm(None, p, p, 1, p, None, 0, None) == 1

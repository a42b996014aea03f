"""ctypes binding of libtomo.so: signatures and status checking only."""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtomo.so")

TOMO_OK = 0
STATUS = {0: "TOMO_OK", 1: "TOMO_ERR_INVALID_ARG", 2: "TOMO_ERR_OOM", 3: "TOMO_ERR_CUDA",
          4: "TOMO_ERR_TIMEOUT", 5: "TOMO_ERR_UNSUPPORTED", 6: "TOMO_ERR_NUMERIC", 7: "TOMO_ERR_IO"}
DTYPES = {"f32": 0, "bf16": 1, "f16": 2}
OP_PROJECT, OP_BACKPROJECT, OP_SIRT, OP_CGLS, OP_SIRT_BB, OP_RESIDUAL = 0, 1, 2, 3, 4, 5
SLICE_MAJOR, INTERLEAVED = 0, 1

# every entry point include/tomo.h declares
EXPORTS = ["tomo_build_matrix", "tomo_matrix_destroy", "tomo_matrix_info", "tomo_matrix_export_rows",
           "tomo_matrix_export_csr",
           "tomo_matrix_export_norms", "tomo_workspace_size", "tomo_project", "tomo_backproject",
           "tomo_sirt", "tomo_cgls", "tomo_cgls_resume", "tomo_cgls_batched", "tomo_cgls_batched_workspace",
           "tomo_sirt_noalloc", "tomo_autotune", "tomo_stream_status", "tomo_sirt_bb",
           "tomo_fubini_create", "tomo_fubini_destroy", "tomo_fubini_project", "tomo_fubini_backproject",
           "tomo_fubini_sirt_bb", "tomo_fubini_normal", "tomo_fubini_sirt_bb_normal", "tomo_tv",
           "tomo_residual_norm", "tomo_status_string", "tomo_last_error"]


class TomoError(RuntimeError):
    def __init__(self, code: int, func: str, msg: str):
        self.code = code
        super().__init__("%s failed with %s: %s" % (func, STATUS.get(code, str(code)), msg))


class Geometry(ctypes.Structure):
    _fields_ = [("n_x", ctypes.c_int32), ("n_y", ctypes.c_int32), ("n_p", ctypes.c_int32),
                ("n_theta", ctypes.c_int32), ("angles", ctypes.c_void_p), ("center", ctypes.c_double)]


class MatrixOpts(ctypes.Structure):
    _fields_ = [("values", ctypes.c_int32), ("no_fp32_sell", ctypes.c_int32), ("drop_csr", ctypes.c_int32),
                ("model", ctypes.c_int32), ("col_blocks", ctypes.c_int32), ("no_at_tiles", ctypes.c_int32),
                ("a_ray_order", ctypes.c_int32), ("reserved", ctypes.c_int32 * 1)]


class Timing(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 4), ("launches", ctypes.c_int64 * 4)]


class ExecOpts(ctypes.Structure):
    _fields_ = [("batch_width", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("format", ctypes.c_int32), ("timeout_s", ctypes.c_float),
                ("timing", ctypes.POINTER(Timing)), ("test_flags", ctypes.c_int32),
                ("async_", ctypes.c_int32), ("recompute_fp32", ctypes.c_int32), ("order", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]


class TuneEntry(ctypes.Structure):
    _fields_ = [("batch_width", ctypes.c_int32), ("format", ctypes.c_int32),
                ("order", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("ms_per_iter", ctypes.c_double), ("slice_iters_per_s", ctypes.c_double)]


class CglsState(ctypes.Structure):
    _fields_ = [("r", ctypes.c_void_p), ("p", ctypes.c_void_p), ("gamma", ctypes.c_void_p),
                ("frozen", ctypes.c_void_p)]


class BbState(ctypes.Structure):
    _fields_ = [("g", ctypes.c_void_p), ("alpha", ctypes.c_void_p), ("frozen", ctypes.c_void_p)]


class Request(ctypes.Structure):
    _fields_ = [("A", ctypes.c_void_p), ("sino", ctypes.c_void_p), ("x", ctypes.c_void_p),
                ("n_z", ctypes.c_int32), ("reserved", ctypes.c_int32), ("resnorm_hist", ctypes.c_void_p),
                ("state_in", ctypes.POINTER(CglsState)), ("state_out", ctypes.POINTER(CglsState))]


class MatrixInfo(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int64), ("cols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("bytes_f32", ctypes.c_int64), ("bytes_lp", ctypes.c_int64),
                ("max_row_len", ctypes.c_int64), ("max_col_len", ctypes.c_int64),
                ("lp_dtype", ctypes.c_int32), ("at_tiles", ctypes.c_int32)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libtomo.so; raises (never falls back) when it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libtomo.so is not built (%s); run `python -m paper_2003_12677_b300.build`" % path)
    lib = ctypes.CDLL(path)
    P, I32, I64, SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
    sigs = {
        "tomo_build_matrix": [ctypes.POINTER(Geometry), ctypes.POINTER(MatrixOpts), P, ctypes.POINTER(P)],
        "tomo_matrix_destroy": [P],
        "tomo_matrix_info": [P, ctypes.POINTER(MatrixInfo)],
        "tomo_matrix_export_rows": [P, I32, I64, I64, P, P, P, I64],
        "tomo_matrix_export_csr": [P, I32, P, P, P, P],
        "tomo_matrix_export_norms": [P, P, P],
        "tomo_workspace_size": [P, I32, I32, ctypes.POINTER(ExecOpts), ctypes.POINTER(SZ)],
        "tomo_project": [P, P, P, I32, I32, ctypes.POINTER(ExecOpts), P, SZ, P],
        "tomo_backproject": [P, P, P, I32, I32, ctypes.POINTER(ExecOpts), P, SZ, P],
        "tomo_sirt": [P, P, P, I32, I32, ctypes.c_float, ctypes.POINTER(ExecOpts), P, SZ, P],
        "tomo_cgls": [P, P, P, I32, I32, I32, P, ctypes.POINTER(ExecOpts), P, SZ, P],
        "tomo_cgls_resume": [P, P, P, I32, I32, I32, P, ctypes.POINTER(CglsState), ctypes.POINTER(CglsState),
                             ctypes.POINTER(ExecOpts), P, SZ, P],
        "tomo_sirt_noalloc": [P, P, P, I32, I32, ctypes.c_float, P],
        "tomo_residual_norm": [P, P, P, I32, P, P, SZ, P],
        "tomo_cgls_batched": [ctypes.POINTER(Request), I32, I32, ctypes.POINTER(ExecOpts), P, SZ, P],
        "tomo_cgls_batched_workspace": [ctypes.POINTER(Request), I32, ctypes.POINTER(ExecOpts),
                                        ctypes.POINTER(SZ)],
        "tomo_autotune": [P, I32, I32, ctypes.POINTER(ExecOpts), ctypes.POINTER(ctypes.c_double),
                          ctypes.POINTER(TuneEntry), I32, ctypes.POINTER(I32), P],
        "tomo_stream_status": [P],
        "tomo_fubini_create": [ctypes.POINTER(Geometry), I32, P, ctypes.POINTER(P)],
        "tomo_fubini_destroy": [P],
        "tomo_fubini_project": [P, P, P, I32, P],
        "tomo_fubini_backproject": [P, P, P, I32, I32, P],
        "tomo_fubini_sirt_bb": [P, P, P, I32, I32, P, P],
        "tomo_fubini_normal": [P, P, P, I32, I32, P],
        "tomo_tv": [P, I32, I32, I32, ctypes.c_float, P, P, P],
        "tomo_fubini_sirt_bb_normal": [P, P, P, I32, I32, P, P],
        "tomo_sirt_bb": [P, P, P, I32, I32, ctypes.c_double, P, ctypes.POINTER(BbState), ctypes.POINTER(BbState),
                         ctypes.POINTER(ExecOpts), P, SZ, P],
    }
    for name, args in sigs.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.tomo_status_string.argtypes = [ctypes.c_int]
    lib.tomo_status_string.restype = ctypes.c_char_p
    lib.tomo_last_error.argtypes = []
    lib.tomo_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def check(code: int, func: str):
    if code != TOMO_OK:
        msg = _lib.tomo_last_error().decode() if _lib is not None else ""
        raise TomoError(code, func, msg)


def status_name(code: int) -> str:
    return load().tomo_status_string(code).decode()


def call(name: str, *args):
    lib = load()
    check(getattr(lib, name)(*args), name)

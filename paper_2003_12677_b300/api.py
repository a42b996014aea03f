"""PyTorch-facing binding of libtomo (argument marshalling only).

Every step runs in the CUDA library; this module checks tensor properties,
passes device pointers and the current CUDA stream, and allocates workspaces
through torch's caching allocator.  There is no CPU path: without a CUDA
device or without libtomo.so every call raises.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Tuple

import numpy as np
import torch

from . import _lib


def _stream() -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t: Optional[torch.Tensor]) -> ctypes.c_void_p:
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _check_tensor(t: torch.Tensor, name: str, shape=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != torch.float32:
        raise TypeError("%s must be float32" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError("%s has shape %s, expected %s" % (name, tuple(t.shape), tuple(shape)))


FORMATS = {"sell": 0, "sell16": 1, "csr": 2, "auto": 3}
FORMAT_NAMES = {v: k for k, v in FORMATS.items()}


def _fmt(fmt) -> int:
    if isinstance(fmt, int):
        return fmt
    if fmt not in FORMATS:
        raise ValueError("fmt must be one of %s" % sorted(FORMATS))
    return FORMATS[fmt]


ORDERS = {"auto": 0, "rows": 1, "tiles": 2, "staged": 3}
_launch = {"order": "auto", "blocks_per_sm": 0}


def set_launch(order: str = "auto", blocks_per_sm: int = 0):
    """Launch shape of the SpMM passes of later calls: the row-group order of
    the A^T passes ("auto", "rows", "tiles" or "staged": the 16-bit passes at
    batch width 16 stream the tiled A^T and stage each tile's detector window
    in shared memory) and the resident blocks per SM (0: all that fit).  "auto" / 0 take tomo_autotune's choice for the slice
    count when there is one.  The results are the same bits either way."""
    if order not in ORDERS:
        raise ValueError("order must be one of %s" % sorted(ORDERS))
    if blocks_per_sm < 0:
        raise ValueError("blocks_per_sm must be >= 0")
    _launch["order"], _launch["blocks_per_sm"] = order, int(blocks_per_sm)


def _exec(batch_width: int = 0, use_graph: bool = True, fmt="sell", timing=None,
          recompute_fp32: bool = False) -> _lib.ExecOpts:
    o = _lib.ExecOpts()
    o.batch_width = batch_width
    o.use_graph = 1 if use_graph else 0
    o.format = _fmt(fmt)
    o.recompute_fp32 = 1 if recompute_fp32 else 0
    o.order = ORDERS[_launch["order"]]
    o.blocks_per_sm = _launch["blocks_per_sm"]
    if timing is not None:
        o.timing = ctypes.pointer(timing)
    return o


def new_timing() -> _lib.Timing:
    """A zeroed tomo_timing to pass as `timing=` (per-kind device ms and launch counts)."""
    return _lib.Timing()


MODELS = {"line": 0, "strip": 1}


class Matrix:
    """A and A^T for one parallel-beam geometry, resident on the current device.

    n_x = n_y = n unless given; n_p defaults to n; angles (radians) default to
    m*pi/n_theta; center defaults to n_p/2.  values in {"f32", "bf16", "f16"}
    also builds the 16-bit encoding used with fmt="sell16"; fp32_sell=False
    skips the FP32 SELL-32 copy and keep_csr=False frees the CSR pair after
    the SELL forms are built (memory for very large geometries).  col_blocks
    > 1 stores the 16-bit A as that many bands of image rows, so that each
    projection pass gathers one band (which can stay in L2); 0 (default)
    chooses enough bands that a band of a 16-slice image batch fits in 48 MB,
    1 keeps one matrix.  at_tiles=False
    skips the tiled copy of the 16-bit A^T (the "staged" order's operand);
    pair_order=False keeps the 16-bit A's rows in ray order instead of groups
    of 2 angles x 4 bins (same results; the pair order gathers faster).
    """

    def __init__(self, n: int, n_theta: int, n_p: Optional[int] = None, n_y: Optional[int] = None,
                 angles=None, center: Optional[float] = None, values: str = "f32", fp32_sell: bool = True,
                 keep_csr: bool = True, model: str = "line", col_blocks: int = 0, at_tiles: bool = True,
                 pair_order: bool = True):
        self._h = None
        lib = _lib.load()
        if not torch.cuda.is_available():
            raise RuntimeError("libtomo needs a CUDA device")
        self.n_x = int(n)
        self.n_y = int(n if n_y is None else n_y)
        self.n_p = int(n if n_p is None else n_p)
        self.n_theta = int(n_theta)
        self._angles = None
        g = _lib.Geometry()
        g.n_x, g.n_y, g.n_p, g.n_theta = self.n_x, self.n_y, self.n_p, self.n_theta
        if angles is not None:
            self._angles = np.ascontiguousarray(np.asarray(angles, np.float64))
            if self._angles.shape != (self.n_theta,):
                raise ValueError("angles must have n_theta entries")
            g.angles = self._angles.ctypes.data
        else:
            g.angles = None
        g.center = float("nan") if center is None else float(center)
        o = _lib.MatrixOpts()
        o.values = _lib.DTYPES[values]
        o.no_fp32_sell = 0 if fp32_sell else 1
        o.drop_csr = 0 if keep_csr else 1
        o.model = MODELS[model]
        o.col_blocks = int(col_blocks)
        o.no_at_tiles = 0 if at_tiles else 1
        o.a_ray_order = 0 if pair_order else 1
        h = ctypes.c_void_p()
        _lib.check(lib.tomo_build_matrix(ctypes.byref(g), ctypes.byref(o), _stream(), ctypes.byref(h)),
                   "tomo_build_matrix")
        self._h = h
        self.values = values
        self.model = model
        info = _lib.MatrixInfo()
        _lib.check(lib.tomo_matrix_info(self._h, ctypes.byref(info)), "tomo_matrix_info")
        self.rows, self.cols, self.nnz = info.rows, info.cols, info.nnz
        self.bytes_f32, self.bytes_lp = info.bytes_f32, info.bytes_lp
        self.max_row_len, self.max_col_len = info.max_row_len, info.max_col_len
        self.has_at_tiles = bool(info.at_tiles)

    @property
    def handle(self) -> ctypes.c_void_p:
        if self._h is None:
            raise RuntimeError("matrix was closed")
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None:
            _lib.load().tomo_matrix_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def export_rows(self, begin: int, end: int, transpose: bool = False) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
        """Rows [begin, end) of A (or A^T) as host (row_ptr int64, col int32, val float32)."""
        lib = _lib.load()
        rp = np.empty(end - begin + 1, np.int64)
        # a first call with capacity 0 fills the row pointers and so the size
        st = lib.tomo_matrix_export_rows(self.handle, int(transpose), begin, end, rp.ctypes.data, None, None, 0)
        if st not in (0, 1):
            _lib.check(st, "tomo_matrix_export_rows")
        need = int(rp[-1])
        col = np.empty(max(need, 1), np.int32)
        val = np.empty(max(need, 1), np.float32)
        _lib.check(lib.tomo_matrix_export_rows(self.handle, int(transpose), begin, end, rp.ctypes.data,
                                               col.ctypes.data, val.ctypes.data, need), "tomo_matrix_export_rows")
        return rp, col[:need], val[:need]

    def export_csr(self, transpose: bool = False):
        """The whole CSR form of A (or of its stored transpose) on the host."""
        n = self.cols if transpose else self.rows
        rp = np.empty(n + 1, np.int64)
        col = np.empty(max(self.nnz, 1), np.int32)
        val = np.empty(max(self.nnz, 1), np.float32)
        _lib.call("tomo_matrix_export_csr", self._h, int(transpose), rp.ctypes.data, col.ctypes.data, val.ctypes.data,
                  _stream())
        return rp, col[:self.nnz], val[:self.nnz]

    def export_norms(self) -> Tuple[np.ndarray, np.ndarray]:
        R = np.empty(self.rows, np.float32)
        C = np.empty(self.cols, np.float32)
        _lib.call("tomo_matrix_export_norms", self.handle, R.ctypes.data, C.ctypes.data)
        return R, C

    def autotune(self, n_z: int, allow_16bit=None) -> dict:
        """Time the SpMM launch shapes for n_z slices on the device (batch
        width, format, row-group order of the A^T pass, then resident blocks
        per SM); the fastest is remembered for calls with batch_width=0,
        fmt="auto" and the default order / blocks.  allow_16bit: include the
        16-bit format (default: when the matrix has one); "only": search it
        alone."""
        if allow_16bit is None:
            allow_16bit = self.values != "f32"
        mode = 2 if allow_16bit == "only" else int(bool(allow_16bit))
        best = _lib.ExecOpts()
        rate = ctypes.c_double()
        table = (_lib.TuneEntry * 64)()
        n = ctypes.c_int32()
        _lib.call("tomo_autotune", self.handle, n_z, mode, ctypes.byref(best), ctypes.byref(rate),
                  table, 64, ctypes.byref(n), _stream())
        names = {1: "rows", 2: "tiles", 3: "staged"}
        rows = [{"batch_width": t.batch_width, "format": FORMAT_NAMES[t.format], "order": names.get(t.order, "auto"),
                 "blocks_per_sm": t.blocks_per_sm, "ms_per_iter": t.ms_per_iter,
                 "slice_iters_per_s": t.slice_iters_per_s} for t in table[:min(n.value, 64)]]
        return {"batch_width": best.batch_width, "format": FORMAT_NAMES[best.format],
                "order": names.get(best.order, "auto"), "blocks_per_sm": best.blocks_per_sm,
                "slice_iters_per_s": rate.value, "table": rows}

    def workspace_size(self, op: int, n_z: int, batch_width: int = 0, fmt="sell") -> int:
        b = ctypes.c_size_t()
        o = _exec(batch_width, True, fmt)
        _lib.call("tomo_workspace_size", self.handle, op, n_z, ctypes.byref(o), ctypes.byref(b))
        return b.value

    def _workspace(self, op, n_z, batch_width, fmt) -> Optional[torch.Tensor]:
        nb = self.workspace_size(op, n_z, batch_width, fmt)
        if nb == 0:
            return None
        return torch.empty(nb, dtype=torch.uint8, device="cuda")


def _nz(t: torch.Tensor, per: int, name: str) -> int:
    if t.numel() % per != 0:
        raise ValueError("%s has %d elements, not a multiple of %d" % (name, t.numel(), per))
    return t.numel() // per


def project(M: Matrix, x: torch.Tensor, out: Optional[torch.Tensor] = None, batch_width: int = 0,
            fmt="sell", interleaved: bool = False, timing=None) -> torch.Tensor:
    """y = A x for a stack of tomograms x (n_z, n_y, n_x) -> sinograms (n_z, n_theta, n_p).

    interleaved=True takes x as (cols, n_z) and returns (rows, n_z)."""
    _check_tensor(x, "x")
    nz = x.shape[-1] if interleaved else _nz(x, M.cols, "x")
    if out is None:
        out = torch.empty((M.rows, nz) if interleaved else (nz, M.n_theta, M.n_p), device=x.device,
                          dtype=torch.float32)
    _check_tensor(out, "out")
    ws = None if interleaved else M._workspace(_lib.OP_PROJECT, nz, batch_width, fmt)
    o = _exec(batch_width, True, fmt, timing)
    _lib.call("tomo_project", M.handle, _ptr(x), _ptr(out), nz, _lib.INTERLEAVED if interleaved else 0,
              ctypes.byref(o), _ptr(ws), 0 if ws is None else ws.numel(), _stream())
    return out


def backproject(M: Matrix, y: torch.Tensor, out: Optional[torch.Tensor] = None, batch_width: int = 0,
                fmt="sell", interleaved: bool = False, timing=None) -> torch.Tensor:
    """x = A^T y for a stack of sinograms y (n_z, n_theta, n_p) -> (n_z, n_y, n_x)."""
    _check_tensor(y, "y")
    nz = y.shape[-1] if interleaved else _nz(y, M.rows, "y")
    if out is None:
        out = torch.empty((M.cols, nz) if interleaved else (nz, M.n_y, M.n_x), device=y.device,
                          dtype=torch.float32)
    _check_tensor(out, "out")
    ws = None if interleaved else M._workspace(_lib.OP_BACKPROJECT, nz, batch_width, fmt)
    o = _exec(batch_width, True, fmt, timing)
    _lib.call("tomo_backproject", M.handle, _ptr(y), _ptr(out), nz, _lib.INTERLEAVED if interleaved else 0,
              ctypes.byref(o), _ptr(ws), 0 if ws is None else ws.numel(), _stream())
    return out


def sirt(M: Matrix, sino: torch.Tensor, iters: int, lam: float = 1.0, x0: Optional[torch.Tensor] = None,
         batch_width: int = 0, fmt="sell", use_graph: bool = True,
         workspace: Optional[torch.Tensor] = None, out: Optional[torch.Tensor] = None, timing=None) -> torch.Tensor:
    """SIRT from x0 (zeros by default): x <- x + lam * C o A^T (R o (b - A x))."""
    _check_tensor(sino, "sino")
    nz = _nz(sino, M.rows, "sino")
    if out is not None:
        x = out
        if x0 is None:
            x.zero_()
        else:
            x.copy_(x0)
    else:
        x = torch.zeros((nz, M.n_y, M.n_x), device=sino.device) if x0 is None else x0.clone()
    _check_tensor(x, "x0", (nz, M.n_y, M.n_x))
    ws = workspace if workspace is not None else M._workspace(_lib.OP_SIRT, nz, batch_width, fmt)
    o = _exec(batch_width, use_graph, fmt, timing)
    _lib.call("tomo_sirt", M.handle, _ptr(sino), _ptr(x), nz, iters, ctypes.c_float(lam), ctypes.byref(o),
              _ptr(ws), 0 if ws is None else ws.numel(), _stream())
    return x


def sirt_noalloc(M: Matrix, sino: torch.Tensor, iters: int, lam: float = 1.0,
                 x0: Optional[torch.Tensor] = None, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """SIRT through tomo_sirt_noalloc: no GPU memory is allocated by the library
    (its scratch is a fixed 16 MiB array inside libtomo).  `out` (or a new
    tensor when None, allocated here by torch) receives the result."""
    _check_tensor(sino, "sino")
    nz = _nz(sino, M.rows, "sino")
    if out is None:
        out = torch.zeros((nz, M.n_y, M.n_x), device=sino.device)
    if x0 is None:
        out.zero_()
    else:
        out.copy_(x0)
    _check_tensor(out, "out", (nz, M.n_y, M.n_x))
    _lib.call("tomo_sirt_noalloc", M.handle, _ptr(sino), _ptr(out), nz, iters, ctypes.c_float(lam), _stream())
    return out


def _state_struct(st: dict) -> _lib.CglsState:
    s = _lib.CglsState()
    s.r, s.p = st["r"].data_ptr(), st["p"].data_ptr()
    s.gamma, s.frozen = st["gamma"].data_ptr(), st["frozen"].data_ptr()
    return s


def cgls(M: Matrix, sino: torch.Tensor, iters: int, recompute_every: int = 0, history: bool = False,
         batch_width: int = 0, fmt="sell", use_graph: bool = True, out: Optional[torch.Tensor] = None,
         workspace: Optional[torch.Tensor] = None, timing=None, resume: Optional[dict] = None,
         return_state: bool = False, recompute_fp32: bool = False):
    """CGLS per slice.  Starts from x0 = 0, or from `resume` (a dict with the
    iterate "x" and the state "r", "p", "gamma", "frozen" as returned with
    return_state=True).  Returns x, then the ||r|| history (iters, n_z) if
    history, then the final state dict if return_state.  recompute_fp32: with
    fmt="sell16", the residual recompute uses the FP32 values of A."""
    _check_tensor(sino, "sino")
    nz = _nz(sino, M.rows, "sino")
    if resume is not None:
        x = resume["x"].clone() if out is None else out.copy_(resume["x"])
    else:
        x = torch.empty((nz, M.n_y, M.n_x), device=sino.device) if out is None else out
    _check_tensor(x, "out", (nz, M.n_y, M.n_x))
    hist = torch.zeros((max(iters, 1), nz), device=sino.device, dtype=torch.float64) if history else None
    ws = workspace if workspace is not None else M._workspace(_lib.OP_CGLS, nz, batch_width, fmt)
    o = _exec(batch_width, use_graph, fmt, timing, recompute_fp32)
    sin = None
    if resume is not None:
        for k in ("r", "p"):
            _check_tensor(resume[k], "resume[%s]" % k)
        sin = _state_struct(resume)
    state = None
    sout = None
    if return_state:
        state = {"r": torch.empty((nz, M.n_theta, M.n_p), device=sino.device),
                 "p": torch.empty((nz, M.n_y, M.n_x), device=sino.device),
                 "gamma": torch.empty(nz, device=sino.device, dtype=torch.float64),
                 "frozen": torch.empty(nz, device=sino.device, dtype=torch.int32)}
        sout = _state_struct(state)
    _lib.call("tomo_cgls_resume", M.handle, _ptr(sino), _ptr(x), nz, iters, recompute_every, _ptr(hist),
              None if sin is None else ctypes.byref(sin), None if sout is None else ctypes.byref(sout),
              ctypes.byref(o), _ptr(ws), 0 if ws is None else ws.numel(), _stream())
    res = [x]
    if history:
        res.append(hist[:iters])
    if return_state:
        state["x"] = x.clone()
        res.append(state)
    return res[0] if len(res) == 1 else tuple(res)


def residual_norm(M: Matrix, sino: torch.Tensor, x: torch.Tensor,
                  workspace: Optional[torch.Tensor] = None) -> torch.Tensor:
    """||b - A x|| per slice (float64, on the device) with FP64 accumulation
    (tomo_residual_norm): the data fit of the FP32-valued operator to ~1e-15."""
    _check_tensor(sino, "sino")
    _check_tensor(x, "x")
    nz = _nz(sino, M.rows, "sino")
    if _nz(x, M.cols, "x") != nz:
        raise ValueError("sino and x hold different slice counts")
    out = torch.empty(nz, dtype=torch.float64, device=sino.device)
    ws = workspace if workspace is not None else M._workspace(_lib.OP_RESIDUAL, nz, 0, "sell")
    _lib.call("tomo_residual_norm", M.handle, _ptr(sino), _ptr(x), nz, _ptr(out), _ptr(ws),
              0 if ws is None else ws.numel(), _stream())
    return out


def sirt_bb(M: Matrix, sino: torch.Tensor, iters: int, first_step: float = 0.0, history: bool = False,
            batch_width: int = 0, fmt="sell", use_graph: bool = True, x0: Optional[torch.Tensor] = None,
            out: Optional[torch.Tensor] = None, workspace: Optional[torch.Tensor] = None, timing=None,
            resume: Optional[dict] = None, return_state: bool = False):
    """SIRT with Hamming preconditioning and the Barzilai-Borwein step (the
    paper's SIRT).  Starts from x0 (default 0) with first step `first_step`
    (0: pi / n_theta, so the first iterate from 0 is the FBP), or continues
    from `resume` (a dict with "x", "g", "alpha", "frozen" as returned with
    return_state=True).  Returns x, then the ||b - A x_k|| history (iters, n_z)
    if history, then the final state dict if return_state."""
    _check_tensor(sino, "sino")
    nz = _nz(sino, M.rows, "sino")
    shape = (nz, M.n_y, M.n_x)
    x = torch.empty(shape, device=sino.device) if out is None else out
    _check_tensor(x, "out", shape)
    if resume is not None:
        x.copy_(resume["x"])
    elif x0 is not None:
        x.copy_(x0)
    else:
        x.zero_()
    hist = torch.zeros((max(iters, 1), nz), device=sino.device, dtype=torch.float64) if history else None
    ws = workspace if workspace is not None else M._workspace(_lib.OP_SIRT_BB, nz, batch_width, fmt)
    o = _exec(batch_width, use_graph, fmt, timing)

    def struct(st):
        b = _lib.BbState()
        b.g, b.alpha, b.frozen = st["g"].data_ptr(), st["alpha"].data_ptr(), st["frozen"].data_ptr()
        return b

    sin = None
    if resume is not None:
        _check_tensor(resume["g"], "resume[g]")
        sin = struct(resume)
    state, sout = None, None
    if return_state:
        state = {"g": torch.empty(shape, device=sino.device),
                 "alpha": torch.empty(nz, device=sino.device, dtype=torch.float64),
                 "frozen": torch.empty(nz, device=sino.device, dtype=torch.int32)}
        sout = struct(state)
    _lib.call("tomo_sirt_bb", M.handle, _ptr(sino), _ptr(x), nz, iters, float(first_step), _ptr(hist),
              None if sin is None else ctypes.byref(sin), None if sout is None else ctypes.byref(sout),
              ctypes.byref(o), _ptr(ws), 0 if ws is None else ws.numel(), _stream())
    res = [x]
    if history:
        res.append(hist[:iters])
    if return_state:
        state["x"] = x.clone()
        res.append(state)
    return res[0] if len(res) == 1 else tuple(res)


def _new_state(M: Matrix, nz: int, device) -> dict:
    return {"r": torch.empty((nz, M.n_theta, M.n_p), device=device),
            "p": torch.empty((nz, M.n_y, M.n_x), device=device),
            "gamma": torch.empty(nz, device=device, dtype=torch.float64),
            "frozen": torch.empty(nz, device=device, dtype=torch.int32)}


def cgls_batched(requests, iters: int, batch_width: int = 16, fmt="sell", history: bool = False,
                 timeout_s: float = 0.0, test_flags: int = 0, workspace: Optional[torch.Tensor] = None,
                 resume=None, return_state: bool = False, asynchronous: bool = False):
    """CGLS for a list of (Matrix, sinogram stack) requests of uneven geometry
    and slice count, all in one persistent launch.  Returns the list of
    reconstructions, then (if history) the list of ||r|| histories
    (iters, n_z), then (if return_state) the list of state dicts (with "x"),
    which `resume` accepts back (one per request, or None).

    asynchronous: return once the launch is queued on the current stream; its
    device status is read later with `stream_status()`.  The returned tensors
    are valid once the stream passes the launch (torch's stream semantics);
    the inputs and the workspace must be kept alive until then (the caching
    allocator keeps them when they stay referenced, or when they were allocated
    on this stream)."""
    reqs = (_lib.Request * len(requests))()
    outs, hists, states, keep = [], [], [], []
    for i, (M, sino) in enumerate(requests):
        _check_tensor(sino, "sino")
        nz = _nz(sino, M.rows, "sino")
        rs = resume[i] if resume is not None else None
        x = rs["x"].clone() if rs is not None else torch.empty((nz, M.n_y, M.n_x), device=sino.device)
        h = torch.zeros((max(iters, 1), nz), device=sino.device, dtype=torch.float64) if history else None
        reqs[i].A = M.handle.value
        reqs[i].sino = sino.data_ptr()
        reqs[i].x = x.data_ptr()
        reqs[i].n_z = nz
        reqs[i].resnorm_hist = 0 if h is None else h.data_ptr()
        if rs is not None:
            sin = _state_struct(rs)
            keep.append(sin)
            reqs[i].state_in = ctypes.pointer(sin)
        if return_state:
            st = _new_state(M, nz, sino.device)
            sout = _state_struct(st)
            keep.append(sout)
            reqs[i].state_out = ctypes.pointer(sout)
            states.append(st)
        outs.append(x)
        hists.append(h)
    o = _exec(batch_width, True, fmt)
    o.timeout_s = timeout_s
    o.test_flags = test_flags
    o.async_ = 1 if asynchronous else 0
    if workspace is None:
        nb = ctypes.c_size_t()
        _lib.call("tomo_cgls_batched_workspace", reqs, len(requests), ctypes.byref(o), ctypes.byref(nb))
        workspace = torch.empty(nb.value, dtype=torch.uint8, device="cuda")
    _lib.call("tomo_cgls_batched", reqs, len(requests), iters, ctypes.byref(o), _ptr(workspace), workspace.numel(),
              _stream())
    res = [outs]
    if history:
        res.append([h[:iters] for h in hists])
    if return_state:
        for st, x in zip(states, outs):
            st["x"] = x.clone()
        res.append(states)
    return res[0] if len(res) == 1 else tuple(res)


def stream_status(stream: Optional[torch.cuda.Stream] = None) -> str:
    """Synchronise `stream` (default: torch's current stream) and return the
    name of the first device status recorded on it since the last call
    ("TOMO_OK", or e.g. "TOMO_ERR_TIMEOUT" from an asynchronous batched
    launch whose bounded barrier wait ran out); the word is reset."""
    s = stream if stream is not None else torch.cuda.current_stream()
    return _lib.status_name(_lib.load().tomo_stream_status(ctypes.c_void_p(s.cuda_stream)))


class Fubini:
    """The Fubini-Radon transform (Fourier slice theorem with Kaiser-Bessel
    gridding, one sparse matrix S and cuFFT) for an n x n image, n_theta
    angles and n_p bins; kw is the window width in grid points."""

    def __init__(self, n: int, n_theta: int, n_p: Optional[int] = None, angles=None,
                 center: Optional[float] = None, kw: int = 6):
        self._h = None
        lib = _lib.load()
        if not torch.cuda.is_available():
            raise RuntimeError("libtomo needs a CUDA device")
        self.n, self.n_theta = int(n), int(n_theta)
        self.n_p = int(n if n_p is None else n_p)
        g = _lib.Geometry()
        g.n_x = g.n_y = self.n
        g.n_p, g.n_theta = self.n_p, self.n_theta
        self._angles = None
        if angles is not None:
            self._angles = np.ascontiguousarray(np.asarray(angles, np.float64))
            if self._angles.shape != (self.n_theta,):
                raise ValueError("angles must have n_theta entries")
            g.angles = self._angles.ctypes.data
        else:
            g.angles = None
        g.center = float("nan") if center is None else float(center)
        h = ctypes.c_void_p()
        _lib.check(lib.tomo_fubini_create(ctypes.byref(g), int(kw), _stream(), ctypes.byref(h)), "tomo_fubini_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None:
            _lib.load().tomo_fubini_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def project(self, x: torch.Tensor) -> torch.Tensor:
        _check_tensor(x, "x")
        nz = _nz(x, self.n * self.n, "x")
        y = torch.empty((nz, self.n_theta, self.n_p), device=x.device)
        _lib.call("tomo_fubini_project", self._h, _ptr(x), _ptr(y), nz, _stream())
        return y

    def backproject(self, y: torch.Tensor, filtered=False) -> torch.Tensor:
        """The exact adjoint of project (filtered=False), iRadon with the ramp
        density (True or "ramp") or with the Hamming-windowed one ("hamming")."""
        _check_tensor(y, "y")
        nz = _nz(y, self.n_theta * self.n_p, "y")
        x = torch.empty((nz, self.n, self.n), device=y.device)
        f = {False: 0, True: 1, "ramp": 1, "hamming": 2}[filtered]
        _lib.call("tomo_fubini_backproject", self._h, _ptr(y), _ptr(x), nz, f, _stream())
        return x

    def sirt_bb(self, sino: torch.Tensor, iters: int, history: bool = False):
        """The paper's SIRT (Hamming preconditioning, BB step) on this operator,
        from x = 0.  Returns x, and the ||b - R x_k|| history if asked."""
        _check_tensor(sino, "sino")
        nz = _nz(sino, self.n_theta * self.n_p, "sino")
        x = torch.empty((nz, self.n, self.n), device=sino.device)
        hist = torch.zeros((max(iters, 1), nz), device=sino.device, dtype=torch.float64) if history else None
        _lib.call("tomo_fubini_sirt_bb", self._h, _ptr(sino), _ptr(x), nz, iters, _ptr(hist), _stream())
        return (x, hist[:iters]) if history else x

    def normal(self, x: torch.Tensor, filtered=False) -> torch.Tensor:
        """N x = backproject(project(x), filtered) for the exact transform, in
        one step (a convolution on the 2n x 2n grid)."""
        _check_tensor(x, "x")
        nz = _nz(x, self.n * self.n, "x")
        y = torch.empty((nz, self.n, self.n), device=x.device)
        f = {False: 0, True: 1, "ramp": 1, "hamming": 2}[filtered]
        _lib.call("tomo_fubini_normal", self._h, _ptr(x), _ptr(y), nz, f, _stream())
        return y

    def sirt_bb_normal(self, sino: torch.Tensor, iters: int, history: bool = False):
        """sirt_bb with the normal operator in one step per iteration.  Returns
        x, and the ||g_k|| history (g_k = c - N x_k) if asked."""
        _check_tensor(sino, "sino")
        nz = _nz(sino, self.n_theta * self.n_p, "sino")
        x = torch.empty((nz, self.n, self.n), device=sino.device)
        hist = torch.zeros((max(iters, 1), nz), device=sino.device, dtype=torch.float64) if history else None
        _lib.call("tomo_fubini_sirt_bb_normal", self._h, _ptr(sino), _ptr(x), nz, iters, _ptr(hist), _stream())
        return (x, hist[:iters]) if history else x


class TomoProject(torch.autograd.Function):
    """y = A x with the stored transpose as the backward: dL/dx = A^T dL/dy."""

    @staticmethod
    def forward(ctx, x: torch.Tensor, M: Matrix, batch_width: int = 0, fmt="sell"):
        ctx.M, ctx.bw, ctx.fmt = M, batch_width, fmt
        return project(M, x.contiguous(), batch_width=batch_width, fmt=fmt)

    @staticmethod
    def backward(ctx, g: torch.Tensor):
        gx = backproject(ctx.M, g.contiguous(), batch_width=ctx.bw, fmt=ctx.fmt)
        return gx, None, None, None


def radon(x: torch.Tensor, M: Matrix, batch_width: int = 0, fmt="sell") -> torch.Tensor:
    """Differentiable forward projection."""
    return TomoProject.apply(x, M, batch_width, fmt)


class TomoTV(torch.autograd.Function):
    """TV_eps(x) summed over slices (tomo_tv); the gradient comes out of the
    same pass and is kept for the backward."""

    @staticmethod
    def forward(ctx, x: torch.Tensor, eps: float):
        x = x.contiguous()
        _check_tensor(x, "x")
        if x.dim() < 2:
            raise ValueError("x must be (..., n_y, n_x)")
        ny, nx = x.shape[-2], x.shape[-1]
        nz = x.numel() // (ny * nx)
        loss = torch.empty(nz, dtype=torch.float64, device=x.device)
        grad = torch.empty_like(x)
        _lib.call("tomo_tv", _ptr(x), nz, ny, nx, float(eps), _ptr(loss), _ptr(grad), _stream())
        ctx.save_for_backward(grad)
        return loss.sum().to(x.dtype)

    @staticmethod
    def backward(ctx, go: torch.Tensor):
        grad, = ctx.saved_tensors
        return go * grad, None


def tv_loss(x: torch.Tensor, eps: float = 1e-3) -> torch.Tensor:
    """Isotropic TV with forward differences (0 on the last row / column),
    summed over the slices of x (..., n_y, n_x); differentiable."""
    return TomoTV.apply(x, eps)

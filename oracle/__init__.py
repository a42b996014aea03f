"""FP64 CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
use this package.  The product library never imports it.  It wraps the plain C
in ``tomo_oracle.c`` (built with gcc, ``-ffp-contract=off``, OpenMP) through
ctypes and promotes every float32 input to float64.

Function map (paper: "Sparse Matrix-Based HPC Tomography"):
  build_matrix      Sec. 2 projection integral, discretised as chord lengths
                    (line model) or as areas in unit-width strips (strip model);
                    Sec. 3.1 CSR sorted by row and column, transpose stored apart
  project / backproject   y = A x, x' = A^T y per slice (Sec. 3, SpMV / SpMM)
  project_mf / backproject_mf   the same without storing A
  sirt / cgls       Sec. 2.1 iterative solvers (classical SIRT, textbook CGLS)
  cgls_mf / cgls_resume_mf      the same CGLS without storing A
  loss_grad         Sec. 2.1 model-based objective with a TV prior
  ramp_response / ramp_filter   Sec. 2.1 preconditioner P = F^dagger D^(1/2) F
                    along the detector, D a Hamming-windowed ramp
  sirt_bb / sirt_bb_resume      Sec. 3.1 SIRT with that preconditioning and the
                    Barzilai-Borwein step; its first step is FBP (Sec. 2.1)
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tomo_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")
_lib = None

_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_dbl = ctypes.c_double
_ptr = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (idempotent)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def build_variant(source: str, out_path: str) -> str:
    """Compile a modified copy of the oracle source (used by the mutation
    tests, which plant mistakes and check that the pins catch them)."""
    src = out_path + ".c"
    with open(src, "w") as f:
        f.write(source)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-fopenmp",
                           "-ffp-contract=off", "-fno-fast-math", src, "-o", out_path, "-lm"])
    return out_path


def _load():
    global _lib
    if _lib is None:
        path = os.environ.get("TOMO_ORACLE_LIB")  # mutation tests load a planted variant
        if not path:
            build()
            path = _LIB
        lib = ctypes.CDLL(path)
        lib.oracle_threads.restype = _i32
        lib.oracle_count.restype = _i64
        lib.oracle_row.restype = _i64
        lib.oracle_weight.restype = _i32
        lib.oracle_loss_grad.restype = _dbl
        lib.oracle_loss_grad_mf.restype = _dbl
        lib.oracle_pixel_row.restype = _i64
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(_ptr)


def threads() -> int:
    return int(_load().oracle_threads())


MODELS = {"line": 0, "strip": 1}


@dataclasses.dataclass
class Geometry:
    nx: int
    ny: int
    n_p: int
    n_theta: int
    angles: Optional[np.ndarray] = None   # radians; None -> m*pi/n_theta
    center: Optional[float] = None         # None -> n_p/2
    model: str = "line"                    # "line" (chord length) | "strip" (area in a unit-width strip)

    def model_id(self) -> int:
        return MODELS[self.model]

    def theta(self) -> np.ndarray:
        if self.angles is not None:
            return np.ascontiguousarray(self.angles, dtype=np.float64)
        t = np.empty(self.n_theta)
        _load().oracle_default_angles(_i32(self.n_theta), _p(t))
        return t

    def c(self) -> float:
        return self.n_p / 2.0 if self.center is None else float(self.center)

    def trig(self):
        th = self.theta()
        cs = np.empty(self.n_theta)
        sn = np.empty(self.n_theta)
        _load().oracle_trig(_i32(self.n_theta), _p(th), _p(cs), _p(sn))
        return cs, sn

    @property
    def rows(self) -> int:
        return self.n_theta * self.n_p

    @property
    def cols(self) -> int:
        return self.nx * self.ny


@dataclasses.dataclass
class CSR:
    rows: int
    cols: int
    row_ptr: np.ndarray   # int64 [rows+1]
    col: np.ndarray       # int32 [nnz]
    val: np.ndarray       # float64 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def transpose(self) -> "CSR":
        lib = _load()
        trp = np.empty(self.cols + 1, np.int64)
        tci = np.empty(self.nnz, np.int32)
        tv = np.empty(self.nnz, np.float64)
        lib.oracle_transpose(_i64(self.rows), _i64(self.cols), _p(self.row_ptr), _p(self.col),
                             _p(self.val), _p(trp), _p(tci), _p(tv))
        return CSR(self.cols, self.rows, trp, tci, tv)

    def dense(self) -> np.ndarray:
        d = np.zeros((self.rows, self.cols))
        for i in range(self.rows):
            for e in range(self.row_ptr[i], self.row_ptr[i + 1]):
                d[i, self.col[e]] += self.val[e]
        return d

    def apply(self, x: np.ndarray) -> np.ndarray:
        """Row-wise SpMV of every slice: x (nz, cols) -> (nz, rows), float64."""
        x = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1, self.cols))
        nz = x.shape[0]
        y = np.empty((nz, self.rows))
        _load().oracle_spmv(_i64(self.rows), _i64(self.cols), _p(self.row_ptr), _p(self.col),
                            _p(self.val), _i32(nz), _p(x), _p(y))
        return y


def weight(g: Geometry, m: int, k: int, ix: int, iy: int) -> Optional[float]:
    cs, sn = g.trig()
    L = _dbl(0.0)
    hit = _load().oracle_weight(_i32(g.nx), _i32(g.ny), _dbl(g.c()), _dbl(cs[m]), _dbl(sn[m]),
                                _i32(k), _i32(ix), _i32(iy), ctypes.byref(L), _i32(g.model_id()))
    return L.value if hit else None


def build_matrix(g: Geometry) -> CSR:
    """A as CSR (int64 row_ptr, int32 col ascending per row, float64 values)."""
    lib = _load()
    cs, sn = g.trig()
    counts = np.empty(g.rows, np.int64)
    nnz = lib.oracle_count(_i32(g.nx), _i32(g.ny), _i32(g.n_p), _i32(g.n_theta), _dbl(g.c()),
                           _p(cs), _p(sn), _p(counts), _i32(g.model_id()))
    rp = np.zeros(g.rows + 1, np.int64)
    np.cumsum(counts, out=rp[1:])
    col = np.empty(nnz, np.int32)
    val = np.empty(nnz, np.float64)
    lib.oracle_fill(_i32(g.nx), _i32(g.ny), _i32(g.n_p), _i32(g.n_theta), _dbl(g.c()),
                    _p(cs), _p(sn), _p(rp), _p(col), _p(val), _i32(g.model_id()))
    return CSR(g.rows, g.cols, rp, col, val)


def row(g: Geometry, i: int):
    """Row i of A by brute force over all pixels: (cols int32, vals float64)."""
    cs, sn = g.trig()
    m, k = divmod(int(i), g.n_p)
    cap = 2 * (g.nx + g.ny) + 8
    col = np.empty(cap, np.int32)
    val = np.empty(cap, np.float64)
    n = _load().oracle_row(_i32(g.nx), _i32(g.ny), _i32(g.n_p), _dbl(g.c()), _dbl(cs[m]),
                           _dbl(sn[m]), _i32(k), _p(col), _p(val), _i64(cap), _i32(g.model_id()))
    assert n <= cap
    return col[:n].copy(), val[:n].copy()


def pixel_row(g: Geometry, j: int):
    """Row j of A^T (one pixel): (ray indices int32, chord lengths float64)."""
    cs, sn = g.trig()
    cap = 3 * g.n_theta + 8
    col = np.empty(cap, np.int32)
    val = np.empty(cap, np.float64)
    n = _load().oracle_pixel_row(_i32(g.nx), _i32(g.ny), _i32(g.n_p), _i32(g.n_theta), _dbl(g.c()), _p(cs), _p(sn),
                                 _i64(int(j)), _p(col), _p(val), _i64(cap), _i32(g.model_id()))
    assert n <= cap
    return col[:n].copy(), val[:n].copy()


def project(A: CSR, x) -> np.ndarray:
    return A.apply(x)


def backproject(AT: CSR, y) -> np.ndarray:
    return AT.apply(y)


def project_mf(g: Geometry, x) -> np.ndarray:
    x = np.ascontiguousarray(np.asarray(x, np.float64).reshape(-1, g.cols))
    nz = x.shape[0]
    cs, sn = g.trig()
    y = np.empty((nz, g.rows))
    _load().oracle_project_mf(_i32(g.nx), _i32(g.ny), _i32(g.n_p), _i32(g.n_theta), _dbl(g.c()),
                              _p(cs), _p(sn), _i32(nz), _p(x), _p(y), _i32(g.model_id()))
    return y


def backproject_mf(g: Geometry, y) -> np.ndarray:
    y = np.ascontiguousarray(np.asarray(y, np.float64).reshape(-1, g.rows))
    nz = y.shape[0]
    cs, sn = g.trig()
    x = np.empty((nz, g.cols))
    _load().oracle_backproject_mf(_i32(g.nx), _i32(g.ny), _i32(g.n_p), _i32(g.n_theta),
                                  _dbl(g.c()), _p(cs), _p(sn), _i32(nz), _p(y), _p(x), _i32(g.model_id()))
    return x


def inv_row_sums(M: CSR) -> np.ndarray:
    out = np.empty(M.rows)
    _load().oracle_inv_row_sums(_i64(M.rows), _p(M.row_ptr), _p(M.val), _p(out))
    return out


def sirt(A: CSR, AT: CSR, b, iters: int, lam: float = 1.0, x0=None) -> np.ndarray:
    b = np.ascontiguousarray(np.asarray(b, np.float64).reshape(-1, A.rows))
    nz = b.shape[0]
    x = np.zeros((nz, A.cols)) if x0 is None else np.array(x0, np.float64).reshape(nz, A.cols)
    x = np.ascontiguousarray(x)
    _load().oracle_sirt(_i64(A.rows), _i64(A.cols), _p(A.row_ptr), _p(A.col), _p(A.val),
                        _p(AT.row_ptr), _p(AT.col), _p(AT.val), _i32(nz), _p(b), _p(x),
                        _i32(iters), _dbl(lam))
    return x


def cgls(A: CSR, AT: CSR, b, iters: int):
    """Returns (x (nz, cols), hist (iters, nz) of ||r|| after each iteration)."""
    b = np.ascontiguousarray(np.asarray(b, np.float64).reshape(-1, A.rows))
    nz = b.shape[0]
    x = np.zeros((nz, A.cols))
    hist = np.zeros((max(iters, 1), nz))
    _load().oracle_cgls(_i64(A.rows), _i64(A.cols), _p(A.row_ptr), _p(A.col), _p(A.val),
                        _p(AT.row_ptr), _p(AT.col), _p(AT.val), _i32(nz), _p(b), _p(x),
                        _i32(iters), _p(hist))
    return x, hist[:iters]


def cgls_resume(A: CSR, AT: CSR, x, r, p, gamma, frozen, iters: int):
    """Continue CGLS from a state; returns (x, r, p, gamma, frozen, hist) in FP64."""
    x = np.ascontiguousarray(np.array(x, np.float64).reshape(-1, A.cols))
    nz = x.shape[0]
    r = np.ascontiguousarray(np.array(r, np.float64).reshape(nz, A.rows))
    p = np.ascontiguousarray(np.array(p, np.float64).reshape(nz, A.cols))
    gamma = np.ascontiguousarray(np.array(gamma, np.float64).reshape(nz))
    frozen = np.ascontiguousarray(np.array(frozen, np.int32).reshape(nz))
    hist = np.zeros((max(iters, 1), nz))
    _load().oracle_cgls_resume(_i64(A.rows), _i64(A.cols), _p(A.row_ptr), _p(A.col), _p(A.val),
                               _p(AT.row_ptr), _p(AT.col), _p(AT.val), _i32(nz), _p(x), _p(r), _p(p),
                               _p(gamma), _p(frozen), _i32(iters), _p(hist))
    return x, r, p, gamma, frozen, hist[:iters]


def cgls_mf(g: Geometry, b, iters: int):
    """cgls without a stored matrix (products generated on the fly, in the
    stored form's summation order, so the iterates are the same bits).
    Returns (x (nz, cols), hist (iters, nz) of ||r|| after each iteration)."""
    b = np.ascontiguousarray(np.asarray(b, np.float64).reshape(-1, g.rows))
    nz = b.shape[0]
    cs, sn = g.trig()
    x = np.zeros((nz, g.cols))
    hist = np.zeros((max(iters, 1), nz))
    _load().oracle_cgls_mf(_i32(g.nx), _i32(g.ny), _i32(g.n_p), _i32(g.n_theta), _dbl(g.c()), _p(cs), _p(sn),
                           _i32(g.model_id()), _i32(nz), _p(b), _p(x), _i32(iters), _p(hist))
    return x, hist[:iters]


def cgls_resume_mf(g: Geometry, x, r, p, gamma, frozen, iters: int):
    """cgls_resume without a stored matrix; returns (x, r, p, gamma, frozen, hist)."""
    x = np.ascontiguousarray(np.array(x, np.float64).reshape(-1, g.cols))
    nz = x.shape[0]
    r = np.ascontiguousarray(np.array(r, np.float64).reshape(nz, g.rows))
    p = np.ascontiguousarray(np.array(p, np.float64).reshape(nz, g.cols))
    gamma = np.ascontiguousarray(np.array(gamma, np.float64).reshape(nz))
    frozen = np.ascontiguousarray(np.array(frozen, np.int32).reshape(nz))
    cs, sn = g.trig()
    hist = np.zeros((max(iters, 1), nz))
    _load().oracle_cgls_resume_mf(_i32(g.nx), _i32(g.ny), _i32(g.n_p), _i32(g.n_theta), _dbl(g.c()), _p(cs),
                                  _p(sn), _i32(g.model_id()), _i32(nz), _p(x), _p(r), _p(p), _p(gamma),
                                  _p(frozen), _i32(iters), _p(hist))
    return x, r, p, gamma, frozen, hist[:iters]


def loss_grad_mf(g: Geometry, x, b, mu: float = 1e-3, eps: float = 1e-3):
    """loss_grad with the matrix-free projector pair (no stored matrix)."""
    x = np.ascontiguousarray(np.asarray(x, np.float64).reshape(-1, g.cols))
    b = np.ascontiguousarray(np.asarray(b, np.float64).reshape(-1, g.rows))
    nz = x.shape[0]
    cs, sn = g.trig()
    grad = np.empty_like(x)
    f = _load().oracle_loss_grad_mf(_i32(g.nx), _i32(g.ny), _i32(g.n_p), _i32(g.n_theta), _dbl(g.c()), _p(cs),
                                    _p(sn), _i32(nz), _p(x), _p(b), _dbl(mu), _dbl(eps), _p(grad),
                                    _i32(g.model_id()))
    return float(f), grad


def loss_grad(A: CSR, AT: CSR, nx: int, ny: int, x, b, mu: float = 1e-3, eps: float = 1e-3):
    """(f, grad) of sum ||A x - b||^2 + mu * TV_eps(x); x (nz, ny*nx), b (nz, rows)."""
    x = np.ascontiguousarray(np.asarray(x, np.float64).reshape(-1, A.cols))
    b = np.ascontiguousarray(np.asarray(b, np.float64).reshape(-1, A.rows))
    nz = x.shape[0]
    g = np.empty_like(x)
    f = _load().oracle_loss_grad(_i64(A.rows), _i64(A.cols), _p(A.row_ptr), _p(A.col), _p(A.val),
                                 _p(AT.row_ptr), _p(AT.col), _p(AT.val), _i32(nx), _i32(ny),
                                 _i32(nz), _p(x), _p(b), _dbl(mu), _dbl(eps), _p(g))
    return float(f), g


# ---------------------------------------------------------------------------
# Preconditioned SIRT with the Barzilai-Borwein step (Sec. 3.1; objective of
# Sec. 2.1).  The filter is written in the Fourier domain exactly as the
# preconditioner is defined (zero-pad, FFT, multiply by D, inverse FFT, crop);
# numpy's FFT serves as the library step.
# ---------------------------------------------------------------------------
def ramp_pad(n_p: int) -> int:
    """Padded length N: the smallest power of two >= 2 n_p (no wrap-around)."""
    n = 1
    while n < 2 * n_p:
        n *= 2
    return n


def ramp_response(n_p: int, window: bool = True) -> np.ndarray:
    """D on the N-point DFT grid (real, even).  D = R * w: R is the DFT of the
    band-limited ramp's sampled kernel (1/4 at 0, -1/(pi n)^2 at odd n, 0 at
    even n, truncated to |n| < N/2), w the Hamming window 0.54 + 0.46 cos(2 pi f)
    at frequency f = min(k, N - k)/N cycles per bin (1 at DC, 0.08 at Nyquist)."""
    N = ramp_pad(n_p)
    n = np.arange(N)
    n = np.where(n < N // 2, n, n - N)          # signed tap index
    h = np.zeros(N)
    h[n == 0] = 0.25
    odd = (n % 2) != 0
    h[odd] = -1.0 / (math.pi * n[odd]) ** 2
    R = np.fft.fft(h).real
    if not window:
        return R
    f = np.abs(n) / N
    return R * (0.54 + 0.46 * np.cos(2.0 * math.pi * f))


def ramp_filter(y, n_p: int, D: Optional[np.ndarray] = None) -> np.ndarray:
    """P^T P y = F^dagger D F y for every projection row (length n_p) of y
    (nz, n_theta * n_p): zero-pad to N, DFT, multiply by D, inverse DFT, crop."""
    D = ramp_response(n_p) if D is None else D
    N = D.shape[0]
    y = np.asarray(y, np.float64)
    nz = y.reshape(-1, y.shape[-1]).shape[0]
    rows = y.reshape(nz, -1, n_p)
    pad = np.zeros(rows.shape[:2] + (N,))
    pad[..., :n_p] = rows
    out = np.fft.ifft(np.fft.fft(pad, axis=-1) * D, axis=-1).real[..., :n_p]
    return out.reshape(nz, -1)


def sirt_bb_resume(A: CSR, AT: CSR, n_p: int, b, x, g_prev, alpha_prev, frozen, iters: int,
                   first_step: Optional[float] = None, D: Optional[np.ndarray] = None):
    """Continue preconditioned BB-SIRT from a state.  Per slice, iteration k:
        r  = b - A x                        (its norm is hist[k])
        gn = A^T P^T P r                    (= -grad of 1/2 ||P (A x - b)||^2)
        alpha = first_step                  when the slice has no previous step
                                            (g_prev None, or its alpha_prev 0 and not frozen)
              = <s,s>/<s,y> (BB1) with s = alpha_prev g_prev, y = -(gn - g_prev)
        x  = x + alpha gn
    A slice is frozen (alpha = 0 from then on) when <s,s> or <s,y> is not
    positive.  Returns (x, gn, alpha, frozen, hist (iters, nz)), all FP64."""
    b = np.asarray(b, np.float64).reshape(-1, A.rows)
    nz = b.shape[0]
    x = np.array(x, np.float64).reshape(nz, A.cols)
    D = ramp_response(n_p) if D is None else D
    alpha = np.array(alpha_prev, np.float64).reshape(nz) if alpha_prev is not None else np.zeros(nz)
    frozen = np.array(frozen, bool).reshape(nz) if frozen is not None else np.zeros(nz, bool)
    gp = None if g_prev is None else np.array(g_prev, np.float64).reshape(nz, A.cols)
    n_theta = A.rows // n_p
    a0 = math.pi / n_theta if first_step is None else float(first_step)
    hist = np.zeros((iters, nz))
    for k in range(iters):
        r = b - project(A, x)
        hist[k] = np.sqrt(np.einsum("ij,ij->i", r, r))
        gn = backproject(AT, ramp_filter(r, n_p, D))
        for s in range(nz):
            if frozen[s]:
                a = 0.0
            elif gp is None or alpha[s] == 0.0:  # no previous step for this slice
                a = a0
            else:
                ss = alpha[s] * alpha[s] * float(np.dot(gp[s], gp[s]))
                sy = -alpha[s] * float(np.dot(gp[s], gn[s] - gp[s]))
                if ss > 0.0 and sy > 0.0:
                    a = ss / sy
                else:
                    a, frozen[s] = 0.0, True
            x[s] += a * gn[s]
            alpha[s] = a
        gp = gn
    return x, gp, alpha, frozen, hist


def sirt_bb(A: CSR, AT: CSR, n_p: int, b, iters: int, first_step: Optional[float] = None,
            D: Optional[np.ndarray] = None):
    """BB-SIRT from x0 = 0: returns (x (nz, cols), hist (iters, nz) of ||b - A x_k||)."""
    b = np.asarray(b, np.float64).reshape(-1, A.rows)
    x0 = np.zeros((b.shape[0], A.cols))
    x, _, _, _, hist = sirt_bb_resume(A, AT, n_p, b, x0, None, None, None, iters, first_step, D)
    return x, hist

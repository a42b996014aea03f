"""Test-side reference recurrences for the CGLS precision pins (test
infrastructure; not the oracle, which stays the C code in oracle/).

`textbook_cgls` is the Hestenes-Stiefel CGLS of Sec. 2.1 written once more
with scipy's sparse products, in a chosen vector precision: float64 gives an
FP64 run with a summation order of its own (scipy sums each row in its own
order and the dots are numpy's pairwise sums), float32 an FP32 run with FP32
vectors and products and FP64 dots and step scalars, which is the arithmetic
of the GPU path.  `lowprec_values` rounds the chord lengths the way the 16-bit
matrix format stores them (value times a(theta) = max(|cos|, |sin|) rounded to
bf16 or f16, times the FP32 factor 1/a(theta) when applied)."""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def csr_pair(A, values=None, dtype=np.float64):
    """(S, S^T) as scipy CSR matrices of the oracle's A (values replaced if given)."""
    v = A.val if values is None else values
    S = sp.csr_matrix((np.asarray(v, dtype), A.col, A.row_ptr), shape=(A.rows, A.cols))
    return S, S.T.tocsr()


def textbook_cgls(S, ST, b, iters, dtype, recompute=0, S_rec=None):
    """Iterates x_1 .. x_iters (float64 copies) of CGLS from x0 = 0 with vectors
    and products in `dtype` and FP64 dots; every `recompute` iterations the
    residual is recomputed as b - S_rec x (S_rec defaults to S)."""
    dt = np.dtype(dtype).type
    S_rec = S if S_rec is None else S_rec

    def dot(u, v):
        return float(np.dot(u.astype(np.float64), v.astype(np.float64)))

    b = np.asarray(b).astype(dt)
    x = np.zeros(S.shape[1], dt)
    r = b.copy()
    s = (ST @ r).astype(dt)
    p = s.copy()
    gamma = dot(s, s)
    out = []
    for k in range(iters):
        q = (S @ p).astype(dt)
        qq = dot(q, q)
        if gamma == 0.0 or qq == 0.0:
            out.append(x.astype(np.float64))
            continue
        alpha = gamma / qq
        x = (x + dt(alpha) * p).astype(dt)
        r = (r - dt(alpha) * q).astype(dt)
        if recompute and (k + 1) % recompute == 0:
            r = (b - (S_rec @ x)).astype(dt)
        s = (ST @ r).astype(dt)
        gnew = dot(s, s)
        beta = gnew / gamma
        gamma = gnew
        p = (s + dt(beta) * p).astype(dt)
        out.append(x.astype(np.float64))
    return out


def _bf16(v):
    """FP64 -> bf16 (8 significand bits), round to nearest even, as float64."""
    m, e = np.frexp(np.asarray(v, np.float64))
    return np.ldexp(np.round(m * 256.0), e - 8)


def lowprec_weights(A, g, kind):
    """(16-bit weights round(L a) as float64, fl32(1/a) of every entry)."""
    cs, sn = g.trig()
    a = np.maximum(np.abs(cs), np.abs(sn))
    ang = np.repeat(np.arange(g.n_theta), g.n_p)                     # angle of every row
    row_a = np.repeat(a[ang], np.diff(A.row_ptr))                     # a of every entry
    scaled = A.val * row_a
    w = _bf16(scaled) if kind == "bf16" else scaled.astype(np.float16).astype(np.float64)
    return w, (1.0 / row_a).astype(np.float32).astype(np.float64)


def lowprec_values(A, g, kind):
    """FP32 values of the 16-bit form: round(L a) to `kind`, times fl32(1/a)."""
    w, sc = lowprec_weights(A, g, kind)
    return (w * sc).astype(np.float32)


def data_fit(S64, b, xs):
    """||b - A x|| (FP64) of every iterate."""
    b = np.asarray(b, np.float64)
    return np.array([np.linalg.norm(b - S64 @ x) for x in xs])


def iters_to_fit(fits, target):
    """First iteration count (1-based) whose data fit is at most target, else None."""
    hit = np.nonzero(np.asarray(fits) <= target)[0]
    return int(hit[0]) + 1 if len(hit) else None

"""FP64 oracle of the Fubini-Radon transform (Sec. 3, Eq. 2) -- test infrastructure only.

The projector of Sec. 3: a 2D Fourier transform of the (deapodized) image, an
interpolation ("gridding") of that spectrum onto the polar grid of (angle,
radial frequency) samples written as one sparse matrix S, then 1D inverse
Fourier transforms along each radial line (the Fourier slice theorem).  The
adjoint runs the same steps transposed; with a density filter on the polar
samples (Sec. 3, the diagonal D) it becomes the filtered backprojection.

Definitions (the readings this oracle fixes where the paper leaves details
open; the same ones bind the CUDA path):
  pixel centres     x_j = ix + 1/2 - n/2, y_j = iy + 1/2 - n/2 (square n x n image)
  detector bins     p_k = k + 1/2 - c
  radial samples    w_q = (q - floor(n_p/2)) / n_p, q = 0 .. n_p - 1
  exact transform   R[u](m, k) = Re( (1/n_p) sum_q e^{+2 pi i w_q p_k}
                                     sum_j u_j e^{-2 pi i w_q (x_j cos t_m + y_j sin t_m)} )
  gridding          oversampled grid G = 2n, Kaiser-Bessel window of width kw
                    grid points, beta = pi sqrt((kw/2)^2 (2 - 1/2)^2 - 0.8),
                    deapodization 1 / phi_hat(x / G) per axis, phi_hat by
                    Gauss-Legendre quadrature of the window.
`fubini_direct` is the exact double sum (small cases); `fubini_project` the
gridding algorithm of Sec. 3 in the steps' own order; `fubini_backproject`
its exact adjoint; `fubini_fbp` the adjoint with the ramp density filter.
numpy's FFT serves as the library step for every Fourier transform.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np
import scipy.sparse


def kb_beta(kw: int, sigma: float = 2.0) -> float:
    """Kaiser-Bessel shape for window width kw grid points at oversampling sigma
    (the choice that minimises aliasing, Beatty et al., IEEE TMI 2005)."""
    return math.pi * math.sqrt((kw / sigma) ** 2 * (sigma - 0.5) ** 2 - 0.8)


def kb_window(t, kw: int, beta: float) -> np.ndarray:
    """phi(t) = I0(beta sqrt(1 - (2t/kw)^2)) on |t| <= kw/2, else 0 (t in grid units)."""
    t = np.asarray(t, np.float64)
    a = 1.0 - (2.0 * t / kw) ** 2
    return np.where(a >= 0.0, np.i0(beta * np.sqrt(np.maximum(a, 0.0))), 0.0)


def kb_hat(s, kw: int, beta: float, nodes: int = 256) -> np.ndarray:
    """phi_hat(s) = int phi(t) cos(2 pi s t) dt by Gauss-Legendre quadrature."""
    xg, wg = np.polynomial.legendre.leggauss(nodes)
    t = xg * (kw / 2.0)
    w = wg * (kw / 2.0)
    s = np.asarray(s, np.float64)
    return np.sum(w * kb_window(t, kw, beta) * np.cos(2.0 * math.pi * np.multiply.outer(s, t)), axis=-1)


@dataclasses.dataclass
class FGeometry:
    n: int                                  # image n x n
    n_p: int
    n_theta: int
    angles: Optional[np.ndarray] = None     # radians; None -> m pi / n_theta
    center: Optional[float] = None          # None -> n_p / 2
    kw: int = 6

    def theta(self) -> np.ndarray:
        if self.angles is not None:
            return np.asarray(self.angles, np.float64)
        return np.arange(self.n_theta, dtype=np.float64) * math.pi / self.n_theta

    def c(self) -> float:
        return self.n_p / 2.0 if self.center is None else float(self.center)

    @property
    def G(self) -> int:
        return 2 * self.n

    def beta(self) -> float:
        return kb_beta(self.kw)

    def omega(self) -> np.ndarray:
        return (np.arange(self.n_p) - self.n_p // 2) / self.n_p

    def pix(self) -> np.ndarray:
        return np.arange(self.n) + 0.5 - self.n / 2.0

    def bins(self) -> np.ndarray:
        return np.arange(self.n_p) + 0.5 - self.c()


def fubini_direct(fg: FGeometry, u) -> np.ndarray:
    """The exact transform as a double sum; u (nz, n*n) -> (nz, n_theta*n_p).  O(n^2 n_theta n_p)."""
    u = np.asarray(u, np.float64).reshape(-1, fg.n, fg.n)
    th = fg.theta()
    x = fg.pix()
    w = fg.omega()
    p = fg.bins()
    E = np.exp(2j * math.pi * np.multiply.outer(w, p)) / fg.n_p          # (q, k)
    out = np.empty((u.shape[0], fg.n_theta, fg.n_p))
    for m in range(fg.n_theta):
        ex = np.exp(-2j * math.pi * np.multiply.outer(w * math.cos(th[m]), x))   # (q, ix)
        ey = np.exp(-2j * math.pi * np.multiply.outer(w * math.sin(th[m]), x))   # (q, iy)
        U = np.einsum("zyx,qx,qy->zq", u, ex, ey)                                  # spectrum on line m
        out[:, m, :] = (U @ E).real
    return out.reshape(u.shape[0], -1)


def gridding_matrix(fg: FGeometry) -> scipy.sparse.csr_matrix:
    """S: (n_theta*n_p) x (G*G), real.  Row (m, q) holds the kw x kw window
    weights phi(ty - ky) phi(tx - kx) around t = G w_q (cos, sin)(t_m), the
    kw grid points k0 .. k0 + kw - 1 per axis with k0 = floor(t - kw/2) + 1;
    the grid index wraps modulo G with a factor -1 per wrap (the half-integer
    pixel centres make the spectrum anti-periodic with period G).  Column
    (ky mod G) * G + (kx mod G); entries of a row in window order (ky, then kx)."""
    G, kw = fg.G, fg.kw
    beta = fg.beta()
    th = fg.theta()
    w = fg.omega()
    tx = G * np.multiply.outer(np.cos(th), w).ravel()          # row r = m * n_p + q
    ty = G * np.multiply.outer(np.sin(th), w).ravel()
    kx = np.floor(tx - kw / 2.0).astype(np.int64)[:, None] + 1 + np.arange(kw)[None, :]   # (rows, kw)
    ky = np.floor(ty - kw / 2.0).astype(np.int64)[:, None] + 1 + np.arange(kw)[None, :]
    wx = kb_window(tx[:, None] - kx, kw, beta)
    wy = kb_window(ty[:, None] - ky, kw, beta)
    sx = np.where(((kx - kx % G) // G) % 2 != 0, -1.0, 1.0)
    sy = np.where(((ky - ky % G) // G) % 2 != 0, -1.0, 1.0)
    vals = (wy * sy)[:, :, None] * (wx * sx)[:, None, :]                       # (rows, a, b)
    cols = (ky % G)[:, :, None] * G + (kx % G)[:, None, :]
    nr = tx.shape[0]
    rows = np.repeat(np.arange(nr), kw * kw)
    return scipy.sparse.csr_matrix((vals.ravel(), (rows, cols.ravel())), shape=(nr, G * G))


def _deapod(fg: FGeometry) -> np.ndarray:
    return 1.0 / kb_hat(fg.pix() / fg.G, fg.kw, fg.beta())


def _grid_phase(fg: FGeometry) -> np.ndarray:
    """e^{2 pi i k (G/2 - 1/2)/G}: turns the DFT over grid indices into the
    transform over the pixel coordinates x = g - G/2 + 1/2."""
    G = fg.G
    return np.exp(2j * math.pi * np.arange(G) * (G / 2.0 - 0.5) / G)


def fubini_project(fg: FGeometry, u, S: Optional[scipy.sparse.csr_matrix] = None) -> np.ndarray:
    """Gridded transform: deapodize, zero-pad to G x G, 2D FFT, grid phase,
    S (polar samples), 1D inverse transform along each radial line, real part."""
    n, G = fg.n, fg.G
    S = gridding_matrix(fg) if S is None else S
    u = np.asarray(u, np.float64).reshape(-1, n, n)
    d = _deapod(fg)
    o = (G - n) // 2
    v = np.zeros((u.shape[0], G, G))
    v[:, o:o + n, o:o + n] = u * d[None, :, None] * d[None, None, :]
    V = np.fft.fft2(v)
    ph = _grid_phase(fg)
    W = V * ph[None, :, None] * ph[None, None, :]
    P = (S @ W.reshape(u.shape[0], -1).T).T.reshape(u.shape[0], fg.n_theta, fg.n_p)   # complex
    E = np.exp(2j * math.pi * np.multiply.outer(fg.omega(), fg.bins())) / fg.n_p      # (q, k)
    return (P @ E).real.reshape(u.shape[0], -1)


def _adjoint_polar(fg: FGeometry, Pq, S) -> np.ndarray:
    """Steps of the adjoint from the polar samples back to the image (real part)."""
    n, G = fg.n, fg.G
    nz = Pq.shape[0]
    Wg = (S.T @ Pq.reshape(nz, -1).T).T.reshape(nz, G, G)
    ph = _grid_phase(fg)
    Wg = Wg * np.conj(ph)[None, :, None] * np.conj(ph)[None, None, :]
    v = np.fft.ifft2(Wg) * (G * G)          # unnormalised inverse DFT = the DFT's adjoint
    o = (G - n) // 2
    d = _deapod(fg)
    return (v[:, o:o + n, o:o + n].real * d[None, :, None] * d[None, None, :]).reshape(nz, -1)


def fubini_backproject(fg: FGeometry, y, S: Optional[scipy.sparse.csr_matrix] = None) -> np.ndarray:
    """Exact adjoint of fubini_project: (nz, n_theta*n_p) -> (nz, n*n)."""
    S = gridding_matrix(fg) if S is None else S
    y = np.asarray(y, np.float64).reshape(-1, fg.n_theta, fg.n_p)
    Eh = np.exp(-2j * math.pi * np.multiply.outer(fg.bins(), fg.omega())) / fg.n_p    # (k, q)
    return _adjoint_polar(fg, y @ Eh, S)


def ramp_density(fg: FGeometry) -> np.ndarray:
    """|w_q| on the radial samples, with the DC sample weighted by the mean of
    |w| over its cell [-1/(2 n_p), 1/(2 n_p)], 1/(4 n_p), instead of 0."""
    d = np.abs(fg.omega())
    d[fg.n_p // 2] = 1.0 / (4.0 * fg.n_p)
    return d


def hamming_density(fg: FGeometry) -> np.ndarray:
    """ramp_density times the Hamming window 0.54 + 0.46 cos(2 pi w_q)."""
    return ramp_density(fg) * (0.54 + 0.46 * np.cos(2.0 * math.pi * fg.omega()))


def fubini_fbp(fg: FGeometry, y, S: Optional[scipy.sparse.csr_matrix] = None,
               density: Optional[np.ndarray] = None) -> np.ndarray:
    """Filtered backprojection (iRadon, Sec. 3): the adjoint with the density
    filter D on the polar samples and the angular weight pi/n_theta, i.e.
    (pi/n_theta) sum_m sum_q D_q (1/n_p) P_m(w_q) e^{2 pi i w_q (x . theta_m)},
    P_m the DFT of projection m (unit bin spacing), D = ramp_density."""
    S = gridding_matrix(fg) if S is None else S
    y = np.asarray(y, np.float64).reshape(-1, fg.n_theta, fg.n_p)
    Eh = np.exp(-2j * math.pi * np.multiply.outer(fg.bins(), fg.omega()))             # (k, q), no 1/n_p
    dens = ramp_density(fg) if density is None else density
    Pq = (y @ Eh) * (dens / fg.n_p)[None, None, :]
    return (math.pi / fg.n_theta) * _adjoint_polar(fg, Pq, S)


def fubini_sirt_bb(fg: FGeometry, b, iters: int, S: Optional[scipy.sparse.csr_matrix] = None):
    """The paper's SIRT (Sec. 3.1: Hamming preconditioning, BB step) on its own
    operator: per slice, r = b - R x (its norm is hist[k]), g = the filtered
    backprojection of r with the Hamming-windowed ramp density
    (= R^T W r for the symmetric PSD sinogram weight W the density defines),
    x += alpha g; alpha = 1 on the first step (so x_1 = the filtered
    backprojection of b), then the BB1 step <s,s>/<s,y> in FP64; a slice whose
    <s,s> or <s,y> is not positive is frozen.  x0 = 0.  Returns (x, hist)."""
    S = gridding_matrix(fg) if S is None else S
    b = np.asarray(b, np.float64).reshape(-1, fg.n_theta * fg.n_p)
    nz = b.shape[0]
    dens = hamming_density(fg)
    x = np.zeros((nz, fg.n * fg.n))
    gp = None
    alpha = np.zeros(nz)
    frozen = np.zeros(nz, bool)
    hist = np.zeros((iters, nz))
    for k in range(iters):
        r = b - fubini_project(fg, x, S)
        hist[k] = np.sqrt(np.einsum("ij,ij->i", r, r))
        g = fubini_fbp(fg, r, S, dens)
        for s_ in range(nz):
            if frozen[s_]:
                a = 0.0
            elif gp is None:
                a = 1.0
            else:
                ss = alpha[s_] * alpha[s_] * float(np.dot(gp[s_], gp[s_]))
                sy = -alpha[s_] * float(np.dot(gp[s_], g[s_] - gp[s_]))
                if ss > 0.0 and sy > 0.0:
                    a = ss / sy
                else:
                    a, frozen[s_] = 0.0, True
            x[s_] += a * g[s_]
            alpha[s_] = a
        gp = g
    return x, hist


# ---------------------------------------------------------------------------
# The normal operator (the Toeplitz route of the paper's outlook, Sec. 5):
# the backprojection (or filtered backprojection) of the exact transform of
# the image, N = R^T W R, in one operation.  The oracle is that composition
# written out with exact double sums; `normal_taps` states the same operator
# entry by entry (a Toeplitz part over pixel differences plus, for even n_p,
# a Hankel part over pixel sums from the unpaired sample w = -1/2).

def normal_weights(fg: FGeometry, filt: int):
    """(kappa, D_q): the weight that the exact adjoint (filt 0: kappa = 1/n_p,
    D = 1) or the filtered backprojection (filt 1 ramp, 2 Hamming-windowed ramp:
    kappa = pi / (n_theta n_p)) puts on polar sample q."""
    if filt == 0:
        return 1.0 / fg.n_p, np.ones(fg.n_p)
    if filt == 1:
        return math.pi / (fg.n_theta * fg.n_p), ramp_density(fg)
    if filt == 2:
        return math.pi / (fg.n_theta * fg.n_p), hamming_density(fg)
    raise ValueError("filt must be 0, 1 or 2")


def fubini_direct_backproject(fg: FGeometry, y, filt: int = 0) -> np.ndarray:
    """Exact adjoint (filt 0) or filtered backprojection (filt 1, 2) of the exact
    transform as a double sum: g_j = kappa Re( sum_m sum_q D_q P_m(w_q)
    e^{2 pi i w_q (x_j cos t_m + y_j sin t_m)} ), P_m(w_q) = sum_k y_mk
    e^{-2 pi i w_q p_k}.  (nz, n_theta*n_p) -> (nz, n*n).  O(n^2 n_theta n_p)."""
    kappa, D = normal_weights(fg, filt)
    y = np.asarray(y, np.float64).reshape(-1, fg.n_theta, fg.n_p)
    th = fg.theta()
    x = fg.pix()
    w = fg.omega()
    Eh = np.exp(-2j * math.pi * np.multiply.outer(fg.bins(), w))        # (k, q)
    out = np.zeros((y.shape[0], fg.n, fg.n))
    for m in range(fg.n_theta):
        P = (y[:, m, :] @ Eh) * (kappa * D)[None, :]                      # (z, q)
        ex = np.exp(2j * math.pi * np.multiply.outer(w * math.cos(th[m]), x))   # (q, ix)
        ey = np.exp(2j * math.pi * np.multiply.outer(w * math.sin(th[m]), x))   # (q, iy)
        out += np.einsum("zq,qx,qy->zyx", P, ex, ey).real
    return out.reshape(y.shape[0], -1)


def fubini_normal(fg: FGeometry, u, filt: int = 0) -> np.ndarray:
    """N u = (exact backprojection, filter filt) of (exact transform of u):
    the definition, (nz, n*n) -> (nz, n*n)."""
    return fubini_direct_backproject(fg, fubini_direct(fg, u), filt)


def normal_taps(fg: FGeometry, d, s, filt: int = 0):
    """Entries of N: N[j, l] = t(x_j - x_l) + h(x_j + x_l), x the pixel
    centres (the differences and sums are integer vectors (dx, dy)).

      t(d) = kappa sum_m sum_q nu_q cos(2 pi w_q (dx cos t_m + dy sin t_m))
      h(s) = kappa (D_q0 / 2) sum_m cos(phi - pi (sx cos t_m + sy sin t_m)),
             phi = 2 pi (1/2 - c), only for even n_p (q0 = 0, w_q0 = -1/2)

    with nu_q = D_q, except nu_q0 = D_q0 / 2 for even n_p.  For real images
    the transform's real part pairs every sample w with -w; the one sample
    without a partner contributes half of its weight shift-invariantly (t) and
    half through the mirror image (h).  d, s: integer arrays (k, 2) of (x, y)
    components.  Returns (t (k,), h (k,))."""
    kappa, D = normal_weights(fg, filt)
    th = fg.theta()
    w = fg.omega()
    nu = D.copy()
    even = fg.n_p % 2 == 0
    if even:
        nu[0] = D[0] / 2.0
    d = np.asarray(d, np.float64).reshape(-1, 2)
    s = np.asarray(s, np.float64).reshape(-1, 2)
    t = np.zeros(d.shape[0])
    h = np.zeros(s.shape[0])
    phi = 2.0 * math.pi * (0.5 - fg.c())
    for m in range(fg.n_theta):
        pd = d[:, 0] * math.cos(th[m]) + d[:, 1] * math.sin(th[m])
        t += np.cos(2.0 * math.pi * np.multiply.outer(pd, w)) @ nu
        if even:
            ps = s[:, 0] * math.cos(th[m]) + s[:, 1] * math.sin(th[m])
            h += np.cos(phi - math.pi * ps)
    return kappa * t, (kappa * D[0] / 2.0 * h if even else h)


def normal_entry_vectors(fg: FGeometry, j, l):
    """(d, s) integer vectors for pixel pairs j, l (flat indices iy * n + ix)."""
    j = np.asarray(j, np.int64)
    l = np.asarray(l, np.int64)
    jx, jy, lx, ly = j % fg.n, j // fg.n, l % fg.n, l // fg.n
    d = np.stack([jx - lx, jy - ly], axis=-1)
    s = np.stack([jx + lx + 1 - fg.n, jy + ly + 1 - fg.n], axis=-1)
    return d, s


def fubini_sirt_bb_normal(fg: FGeometry, b, iters: int, S: Optional[scipy.sparse.csr_matrix] = None):
    """The paper's SIRT (Sec. 3.1) with the normal operator in one step: per
    slice, c = the Hamming-filtered backprojection of b (gridded, computed once),
    g_k = c - N x_k (N = fubini_normal with the Hamming filter; ||g_k|| is
    hist[k]), x += alpha g with alpha = 1 on the first step and the BB1 step
    <s,s>/<s,y> after it, in FP64; a slice whose <s,s> or <s,y> is not positive
    is frozen.  x0 = 0.  Returns (x, hist)."""
    S = gridding_matrix(fg) if S is None else S
    b = np.asarray(b, np.float64).reshape(-1, fg.n_theta * fg.n_p)
    nz = b.shape[0]
    c = fubini_fbp(fg, b, S, hamming_density(fg))
    x = np.zeros((nz, fg.n * fg.n))
    gp = None
    alpha = np.zeros(nz)
    frozen = np.zeros(nz, bool)
    hist = np.zeros((iters, nz))
    for k in range(iters):
        g = c - fubini_normal(fg, x, 2)
        hist[k] = np.sqrt(np.einsum("ij,ij->i", g, g))
        for s_ in range(nz):
            if frozen[s_]:
                a = 0.0
            elif gp is None:
                a = 1.0
            else:
                ss = alpha[s_] * alpha[s_] * float(np.dot(gp[s_], gp[s_]))
                sy = -alpha[s_] * float(np.dot(gp[s_], g[s_] - gp[s_]))
                if ss > 0.0 and sy > 0.0:
                    a = ss / sy
                else:
                    a, frozen[s_] = 0.0, True
            x[s_] = x[s_] + a * g[s_]
            alpha[s_] = a
        gp = g
    return x, hist

"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test states what fixes the expected value: a special angle where the chord
lengths are known exactly, an independent clipping algorithm, a closed-form
projection, a conservation law, the definition of the transpose, a spectral
closed form of the SIRT recurrence, the Krylov-subspace minimiser that CGLS
must reproduce, or finite differences of the objective.
"""
import math

import numpy as np
import pytest
import scipy.linalg
import scipy.sparse

import oracle
from paper_2003_12677_b300 import inputs


# ---------------------------------------------------------------------------
# independent chord-length reference: Liang-Barsky clipping of the ray
# ---------------------------------------------------------------------------

def clip_length(theta, p, xc, yc):
    """Length of {x cos t + y sin t = p} inside the unit square centred (xc, yc).

    The line is parametrised as p*(cos, sin) + s*(-sin, cos) and the s-range
    clipped against the four slabs (Liang & Barsky, 1984)."""
    c, s_ = math.cos(theta), math.sin(theta)
    x0, y0 = p * c, p * s_
    dx, dy = -s_, c
    lo, hi = -1e300, 1e300
    for d, o, a, b in ((dx, x0, xc - 0.5, xc + 0.5), (dy, y0, yc - 0.5, yc + 0.5)):
        if abs(d) < 1e-300:
            if o < a or o > b:
                return 0.0
            continue
        t1, t2 = (a - o) / d, (b - o) / d
        lo, hi = max(lo, min(t1, t2)), min(hi, max(t1, t2))
    return max(0.0, hi - lo)


@pytest.mark.parametrize("nx,ny,n_p,center,angles", [
    (8, 8, 8, None, [0.0, math.pi / 4, math.pi / 2, 0.3, 1.1, 2.0, 2.9, 3.0]),
    (8, 8, 11, 5.3, [0.05, 0.7, 1.5707, 1.6, 2.356194490192345, 3.1]),
    (7, 9, 12, None, list(np.random.default_rng(3).uniform(0, math.pi, 10))),
])
def test_weights_match_clipping(nx, ny, n_p, center, angles):
    g = oracle.Geometry(nx, ny, n_p, len(angles), np.array(angles), center)
    A = oracle.build_matrix(g)
    cs, sn = g.trig()
    c = g.c()
    dense = A.dense()
    checked = 0
    for m, th in enumerate(g.theta()):
        a = max(abs(cs[m]), abs(sn[m]))
        e = min(abs(cs[m]), abs(sn[m]))
        h = 0.5 * (a + e)
        for k in range(n_p):
            p = k + 0.5 - c
            for iy in range(ny):
                for ix in range(nx):
                    xc, yc = ix + 0.5 - nx / 2, iy + 0.5 - ny / 2
                    delta = abs(p - (xc * cs[m] + yc * sn[m]))
                    if abs(delta - h) < 1e-9:
                        continue  # line through a corner / along an edge
                    ref = clip_length(th, p, xc, yc)
                    got = dense[m * n_p + k, iy * nx + ix]
                    assert abs(got - ref) < 1e-12, (m, k, ix, iy, got, ref)
                    checked += 1
    assert checked > 0.9 * A.rows * A.cols


def test_structure_invariants():
    g = oracle.Geometry(32, 32, 40, 17, center=19.25)
    A = oracle.build_matrix(g)
    rp, col, val = A.row_ptr, A.col, A.val
    assert rp[0] == 0 and np.all(np.diff(rp) >= 0)
    for i in range(A.rows):
        cc = col[rp[i]:rp[i + 1]]
        assert np.all(np.diff(cc) > 0)  # strictly ascending, no duplicates
    assert np.all(val > 0) and np.all(val <= math.sqrt(2) + 1e-15)
    assert col.min() >= 0 and col.max() < A.cols
    # the brute-force row walk over every pixel gives the same rows
    for i in list(range(0, A.rows, 37)) + [A.rows - 1]:
        c2, v2 = oracle.row(g, i)
        np.testing.assert_array_equal(c2, col[rp[i]:rp[i + 1]])
        np.testing.assert_array_equal(v2, val[rp[i]:rp[i + 1]])


def test_theta_zero_is_column_sum():
    """theta = 0: ray k is the pixel column ix = k; every chord is exactly 1."""
    n = 16
    g = oracle.Geometry(n, n, n, 4)
    A = oracle.build_matrix(g)
    for k in range(n):
        cc = A.col[A.row_ptr[k]:A.row_ptr[k + 1]]
        vv = A.val[A.row_ptr[k]:A.row_ptr[k + 1]]
        np.testing.assert_array_equal(cc, np.arange(n) * n + k)
        assert np.all(vv == 1.0)


def test_theta_half_pi_is_row_sum():
    """theta = pi/2 (m = 1 of 2 angles): ray k is the pixel row iy = k, chord 1."""
    n = 16
    g = oracle.Geometry(n, n, n, 2)
    A = oracle.build_matrix(g)
    for k in range(n):
        i = n + k
        cc = A.col[A.row_ptr[i]:A.row_ptr[i + 1]]
        vv = A.val[A.row_ptr[i]:A.row_ptr[i + 1]]
        np.testing.assert_array_equal(cc, k * n + np.arange(n))
        assert np.all(vv == 1.0)


def _disk_error(n, n_theta=24):
    r = 0.3 * n
    g = oracle.Geometry(n, n, n, n_theta)
    A = oracle.build_matrix(g)
    x = (np.arange(n) + 0.5 - n / 2)
    X, Y = np.meshgrid(x, x)
    img = (X * X + Y * Y <= r * r).astype(np.float64)
    y = A.apply(img.reshape(1, -1)).reshape(n_theta, n)
    s = np.arange(n) + 0.5 - n / 2
    ref = np.where(np.abs(s) < r, 2 * np.sqrt(np.maximum(r * r - s * s, 0)), 0.0)
    ref = np.broadcast_to(ref, y.shape)
    return np.linalg.norm(y - ref) / np.linalg.norm(ref)


def test_uniform_disk_closed_form():
    """Centred disk of radius r: every projection is 2 sqrt(r^2 - s^2)."""
    e64, e128, e256 = _disk_error(64), _disk_error(128), _disk_error(256)
    assert e128 < 3e-2
    assert e256 < e128 < e64          # pixelisation error falls as n doubles


def test_gaussian_blob_closed_form():
    """exp(-r^2/2 sigma^2) projects to sqrt(2 pi) sigma exp(-s^2/2 sigma^2)."""
    n, sig, nt = 96, 6.0, 12
    g = oracle.Geometry(n, n, n, nt)
    A = oracle.build_matrix(g)
    x = np.arange(n) + 0.5 - n / 2
    X, Y = np.meshgrid(x, x)
    img = np.exp(-(X * X + Y * Y) / (2 * sig * sig))
    y = A.apply(img.reshape(1, -1)).reshape(nt, n)
    ref = math.sqrt(2 * math.pi) * sig * np.exp(-x * x / (2 * sig * sig))
    err = np.linalg.norm(y - ref[None, :]) / np.linalg.norm(np.broadcast_to(ref, y.shape))
    assert err < 1e-3


def test_ellipse_closed_form():
    """Random ellipses: the discrete projection approaches the analytic one."""
    errs = []
    for n in (64, 128, 256):
        rng = np.random.default_rng(7)
        ell = inputs.random_ellipses(n, rng, 6)
        g = oracle.Geometry(n, n, n, 16)
        A = oracle.build_matrix(g)
        y = A.apply(inputs.rasterize(ell, n, n).reshape(1, -1)).reshape(16, n)
        ref = inputs.project_ellipses(ell, g.theta(), n)
        errs.append(np.linalg.norm(y - ref) / np.linalg.norm(ref))
    assert errs[2] < errs[0] and errs[1] < 5e-2


def test_mass_conservation():
    """sum_k (A x)_{m,k} = sum_j x_j: exact at theta = 0 and pi/2 (unit chords),
    within the unit-spacing sampling error of the chord trapezoid elsewhere."""
    n = 128
    nt = 8
    g = oracle.Geometry(n, n, n, nt)
    A = oracle.build_matrix(g)
    ell = inputs.random_ellipses(n, np.random.default_rng(11))
    img = inputs.rasterize(ell, n, n)
    y = A.apply(img.reshape(1, -1)).reshape(nt, n)
    tot = img.sum()
    rel = np.abs(y.sum(axis=1) - tot) / tot
    assert rel[0] < 1e-13 and rel[nt // 2] < 1e-13
    assert rel.max() < 1e-3


@pytest.mark.parametrize("model", ["line", "strip"])
def test_transpose_is_exact_transpose(model):
    g = oracle.Geometry(24, 20, 30, 13, center=14.6, model=model)
    A = oracle.build_matrix(g)
    AT = A.transpose()
    S = scipy.sparse.csr_matrix((A.val, A.col, A.row_ptr), shape=(A.rows, A.cols))
    T = S.T.tocsr()
    T.sort_indices()
    np.testing.assert_array_equal(AT.row_ptr, T.indptr)
    np.testing.assert_array_equal(AT.col, T.indices)
    np.testing.assert_array_equal(AT.val, T.data)


@pytest.mark.parametrize("model", ["line", "strip"])
def test_adjoint_identity_fp64(model):
    g = oracle.Geometry(40, 40, 44, 31, model=model)
    A = oracle.build_matrix(g)
    AT = A.transpose()
    rng = np.random.default_rng(5)
    x = rng.standard_normal((3, A.cols))
    y = rng.standard_normal((3, A.rows))
    lhs = np.sum(A.apply(x) * y)
    rhs = np.sum(x * AT.apply(y))
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs) * 10


@pytest.mark.parametrize("model", ["line", "strip"])
def test_pixel_rows_are_the_transpose_rows(model):
    g = oracle.Geometry(30, 26, 34, 19, center=16.4, model=model)
    A = oracle.build_matrix(g)
    AT = A.transpose()
    for j in list(range(0, A.cols, 53)) + [0, A.cols - 1]:
        c, v = oracle.pixel_row(g, j)
        np.testing.assert_array_equal(c, AT.col[AT.row_ptr[j]:AT.row_ptr[j + 1]])
        np.testing.assert_array_equal(v, AT.val[AT.row_ptr[j]:AT.row_ptr[j + 1]])


def test_matrix_free_loss_grad_equals_stored():
    g = oracle.Geometry(20, 20, 22, 15)
    A = oracle.build_matrix(g)
    AT = A.transpose()
    rng = np.random.default_rng(21)
    x = rng.random((2, A.cols))
    b = rng.random((2, A.rows))
    f1, g1 = oracle.loss_grad(A, AT, 20, 20, x, b)
    f2, g2 = oracle.loss_grad_mf(g, x, b)
    assert f1 == f2
    np.testing.assert_array_equal(g1, g2)


@pytest.mark.parametrize("model", ["line", "strip"])
def test_matrix_free_equals_stored(model):
    g = oracle.Geometry(33, 33, 35, 21, center=17.2, model=model)
    A = oracle.build_matrix(g)
    AT = A.transpose()
    rng = np.random.default_rng(9)
    x = rng.random((2, A.cols))
    y = rng.random((2, A.rows))
    np.testing.assert_array_equal(oracle.project_mf(g, x), A.apply(x))
    np.testing.assert_array_equal(oracle.backproject_mf(g, y), AT.apply(y))


# ---------------------------------------------------------------------------
# SIRT: spectral closed form of the preconditioned Landweber recurrence
# ---------------------------------------------------------------------------

def _inv(v):
    """Reciprocal with 1/0 -> 0 (rays that miss the image carry no weight)."""
    out = np.zeros_like(v)
    out[v != 0] = 1.0 / v[v != 0]
    return out


def _small_system(n=8, nt=16, n_p=12, seed=0):
    g = oracle.Geometry(n, n, n_p, nt)
    A = oracle.build_matrix(g)
    return g, A, A.transpose()


def test_sirt_spectral_closed_form():
    """x_k = C^1/2 V f_k(mu) V^T lam C^1/2 A^T R b, with C^1/2 H C^1/2 = V mu V^T,
    H = A^T R A and f_k(mu) = (1 - (1 - lam mu)^k)/(lam mu) (k when mu = 0)."""
    g, A, AT = _small_system()
    D = A.dense()
    R = _inv(D.sum(axis=1))
    C = _inv(D.sum(axis=0))
    rng = np.random.default_rng(1)
    b = rng.random(A.rows)
    lam = 0.9
    H = D.T @ (R[:, None] * D)
    Ch = np.sqrt(C)
    S = Ch[:, None] * H * Ch[None, :]
    mu, V = scipy.linalg.eigh(S)
    gvec = lam * Ch * (D.T @ (R * b))
    for k in (1, 2, 7, 40):
        lm = lam * mu
        fk = np.where(np.abs(lm) > 1e-14, (1 - (1 - lm) ** k) / np.where(lm == 0, 1, lm), k)
        ref = Ch * (V @ (fk * (V.T @ gvec)))
        got = oracle.sirt(A, AT, b[None], k, lam)[0]
        assert np.max(np.abs(got - ref)) <= 1e-11 * max(1.0, np.max(np.abs(ref)))


def test_sirt_limit_is_weighted_least_squares():
    """The SIRT fixed point solves min ||R^1/2 (A x - b)|| (unique: full rank)."""
    g, A, AT = _small_system()
    D = A.dense()
    assert np.linalg.matrix_rank(D) == A.cols
    R = _inv(D.sum(axis=1))
    rng = np.random.default_rng(2)
    b = rng.random(A.rows)
    ref = np.linalg.lstsq(np.sqrt(R)[:, None] * D, np.sqrt(R) * b, rcond=None)[0]
    got = oracle.sirt(A, AT, b[None], 100000, 1.0)[0]
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-8


# ---------------------------------------------------------------------------
# CGLS: the k-th iterate minimises ||A x - b|| over the Krylov space
# ---------------------------------------------------------------------------

def _krylov_min(D, b, k):
    H = D.T @ D
    q = D.T @ b
    Q = np.zeros((D.shape[1], k))
    v = q / np.linalg.norm(q)
    for j in range(k):
        for _ in range(2):  # Gram-Schmidt twice
            v = v - Q[:, :j] @ (Q[:, :j].T @ v)
        v = v / np.linalg.norm(v)
        Q[:, j] = v
        v = H @ v
    y = np.linalg.lstsq(D @ Q, b, rcond=None)[0]
    return Q @ y


def test_cgls_krylov_minimiser():
    g, A, AT = _small_system()
    D = A.dense()
    rng = np.random.default_rng(4)
    b = rng.random((2, A.rows))
    for k in (1, 2, 3, 5, 8, 10):
        x, hist = oracle.cgls(A, AT, b, k)
        for s in range(2):
            ref = _krylov_min(D, b[s], k)
            assert np.linalg.norm(x[s] - ref) <= 1e-9 * np.linalg.norm(ref)
            assert abs(hist[-1, s] - np.linalg.norm(D @ ref - b[s])) <= 1e-9 * np.linalg.norm(b[s])


def test_cgls_reaches_lstsq():
    g, A, AT = _small_system()
    D = A.dense()
    b = np.random.default_rng(6).random(A.rows)
    ref = np.linalg.lstsq(D, b, rcond=None)[0]
    x, _ = oracle.cgls(A, AT, b[None], 200)
    assert np.linalg.norm(x[0] - ref) <= 1e-6 * np.linalg.norm(ref)


def test_cgls_resume_continues_the_same_recurrence():
    """The cold state (x = 0, r = b, p = A^T b, gamma = |A^T b|^2) resumed for
    k iterations is the k-iteration run bit for bit, and resuming that state
    for m more is the (k+m)-iteration run bit for bit; the state's residual
    equals b - A x to rounding."""
    g, A, AT = _small_system()
    D = A.dense()
    b = np.random.default_rng(10).random((2, A.rows))
    x12, h12 = oracle.cgls(A, AT, b, 12)
    x5, _ = oracle.cgls(A, AT, b, 5)
    s0 = AT.apply(b)
    gamma0 = np.zeros(2)
    for z in range(2):          # sequential sum, as the oracle accumulates it
        acc = 0.0
        for v in s0[z]:
            acc += v * v
        gamma0[z] = acc
    xs, rs, ps, gs, fs, _ = oracle.cgls_resume(A, AT, np.zeros((2, A.cols)), b, s0, gamma0,
                                               np.zeros(2, np.int32), 5)
    np.testing.assert_array_equal(xs, x5)
    np.testing.assert_allclose(rs, b - x5 @ D.T, rtol=0, atol=1e-12 * np.abs(b).max())
    xr, _, _, _, _, hr = oracle.cgls_resume(A, AT, xs, rs, ps, gs, fs, 7)
    np.testing.assert_array_equal(xr, x12)
    np.testing.assert_array_equal(hr, h12[5:])


@pytest.mark.parametrize("n,nt,n_p,center", [(16, 20, 16, None), (13, 8, 17, 7.3), (24, 6, 30, None)])
def test_quarter_turn_symmetry(n, nt, n_p, center):
    """The ray of angle theta + pi/2 meets pixel (ix, iy) exactly as the ray of
    theta with the same bin meets pixel (iy, n - 1 - ix): the square grid and
    the detector line are symmetric under a quarter turn.  So with the default
    angles and an even n_theta, row (m + n_theta/2, k) of A is row (m, k) with
    its columns turned; the FP64 evaluation of the two angles' cosines and
    sines differs in the last bits, which moves the values by ~1e-13 and can
    flip only entries of length ~0 (a line through a pixel corner)."""
    g = oracle.Geometry(n, n, n_p, nt, None, center)
    D = oracle.build_matrix(g).dense()
    half = nt // 2 * n_p
    rho = np.array([(n - 1 - (j % n)) * n + (j // n) for j in range(n * n)])
    turned = D[:half][:, rho]
    assert np.abs(D[half:] - turned).max() < 1e-12
    flipped = (D[half:] != 0) != (turned != 0)
    assert np.all(np.maximum(D[half:], turned)[flipped] < 1e-12)


def test_cgls_matrix_free_equals_stored():
    """The matrix-free CGLS (products generated on the fly) takes the same
    steps in the same summation order as the stored form: bit for bit, from
    zero and from a resumed state, on a non-square grid with an odd detector."""
    g = oracle.Geometry(13, 11, 17, 9)
    A = oracle.build_matrix(g)
    AT = A.transpose()
    b = np.random.default_rng(12).random((3, A.rows))
    x1, h1 = oracle.cgls(A, AT, b, 7)
    x2, h2 = oracle.cgls_mf(g, b, 7)
    np.testing.assert_array_equal(x1, x2)
    np.testing.assert_array_equal(h1, h2)
    st = [x1, b - A.apply(x1), np.random.default_rng(13).random((3, A.cols)), np.ones(3), np.zeros(3, np.int32)]
    for u, v in zip(oracle.cgls_resume(A, AT, *st, 4), oracle.cgls_resume_mf(g, *st, 4)):
        np.testing.assert_array_equal(u, v)


def test_cgls_zero_rhs_freezes():
    g, A, AT = _small_system()
    x, hist = oracle.cgls(A, AT, np.zeros((1, A.rows)), 5)
    assert np.all(x == 0) and np.all(hist == 0)


# ---------------------------------------------------------------------------
# loss / gradient of ||A x - b||^2 + mu TV_eps(x)
# ---------------------------------------------------------------------------

def test_tv_value_hand_computed():
    """2x2 image [[0,1],[2,3]] with data term 0: TV = sqrt(5+e^2) + sqrt(4+e^2)
    + sqrt(1+e^2) + e (forward differences, zero on the last row / column)."""
    g = oracle.Geometry(2, 2, 3, 3)
    A = oracle.build_matrix(g)
    AT = A.transpose()
    x = np.array([[0.0, 1.0, 2.0, 3.0]])
    b = A.apply(x)
    mu, eps = 0.5, 0.1
    f, grad = oracle.loss_grad(A, AT, 2, 2, x, b, mu, eps)
    ref = mu * (math.sqrt(5 + eps ** 2) + math.sqrt(4 + eps ** 2) + math.sqrt(1 + eps ** 2) + eps)
    assert abs(f - ref) < 1e-14


def test_gradient_finite_differences():
    n = 12
    g = oracle.Geometry(n, n, 14, 10)
    A = oracle.build_matrix(g)
    AT = A.transpose()
    rng = np.random.default_rng(8)
    x = rng.random((2, A.cols))
    b = rng.random((2, A.rows))
    f0, grad = oracle.loss_grad(A, AT, n, n, x, b, 1e-3, 1e-3)
    h = 1e-3
    for _ in range(64):
        v = rng.standard_normal(x.shape)
        v /= np.linalg.norm(v)
        fp, _ = oracle.loss_grad(A, AT, n, n, x + h * v, b, 1e-3, 1e-3)
        fm, _ = oracle.loss_grad(A, AT, n, n, x - h * v, b, 1e-3, 1e-3)
        fd = (fp - fm) / (2 * h)
        an = float(np.sum(grad * v))
        assert abs(fd - an) <= 1e-7 * max(1.0, abs(an))


# ---------------------------------------------------------------------------
# preconditioned SIRT with the Barzilai-Borwein step (Sec. 3.1 / Sec. 2.1)
# ---------------------------------------------------------------------------

def ramlak(n):
    """Band-limited ramp sampled at unit spacing (Kak & Slaney, Ch. 3):
    1/4 at 0, 0 at even n, -1/(pi n)^2 at odd n."""
    if n == 0:
        return 0.25
    return 0.0 if n % 2 == 0 else -1.0 / (math.pi * n) ** 2


@pytest.mark.parametrize("n_p", [8, 13, 64])
def test_unwindowed_filter_is_the_ramlak_convolution(n_p):
    """Without the window, filtering a unit impulse at bin j gives the sampled
    band-limited ramp h[k - j] at every bin k (closed form, no wrap-around)."""
    D = oracle.ramp_response(n_p, window=False)
    for j in (0, n_p // 2, n_p - 1):
        y = np.zeros((1, n_p))
        y[0, j] = 1.0
        out = oracle.ramp_filter(y, n_p, D)[0]
        ref = np.array([ramlak(k - j) for k in range(n_p)])
        np.testing.assert_allclose(out, ref, rtol=0, atol=1e-15)


@pytest.mark.parametrize("n_p", [8, 100, 512])
def test_ramp_response_is_a_ramp_with_hamming_ends(n_p):
    """The unwindowed response approximates |f| (cycles per bin) to O(1/N),
    and the Hamming window is 1 at DC and 0.08 at the Nyquist frequency."""
    R = oracle.ramp_response(n_p, window=False)
    D = oracle.ramp_response(n_p)
    N = R.shape[0]
    assert N >= 2 * n_p and N & (N - 1) == 0
    f = np.minimum(np.arange(N), N - np.arange(N)) / N
    assert np.abs(R - f).max() <= 0.5 / N
    assert np.all(R > 0)
    assert D[0] == pytest.approx(R[0], rel=1e-15)
    assert D[N // 2] == pytest.approx(0.08 * R[N // 2], rel=1e-12)


def test_bb_first_step_is_fbp_of_a_disk():
    """Sec. 2.1: FBP is the first step of the preconditioned steepest descent
    from 0.  With the analytic projections of a centred uniform disk (density 1,
    radius 0.3 n), the first BB-SIRT iterate is 1 inside the disk to 1% and
    near 0 outside it within the field of view (the square's corners project
    past the detector at some angles and are left out)."""
    n, nt = 128, 180
    g = oracle.Geometry(n, n, n, nt)
    A = oracle.build_matrix(g)
    AT = A.transpose()
    R = 0.3 * n
    p = np.arange(n) + 0.5 - n / 2
    b = np.tile(np.where(np.abs(p) < R, 2 * np.sqrt(np.maximum(R * R - p * p, 0.0)), 0.0), nt)
    x1, hist = oracle.sirt_bb(A, AT, n, b[None], 1)
    c = np.arange(n) + 0.5 - n / 2
    X, Y = np.meshgrid(c, c)
    rr = np.sqrt(X ** 2 + Y ** 2).ravel()
    assert abs(x1[0][rr < 0.8 * R].mean() - 1.0) < 0.01
    assert x1[0][rr < 0.8 * R].std() < 0.02
    ring = (rr > 1.3 * R) & (rr < 0.5 * n)  # outside the disk, inside the detector's field of view
    assert np.abs(x1[0][ring]).mean() < 0.01
    assert hist[0, 0] == pytest.approx(np.linalg.norm(b))


def test_bb_converges_to_preconditioned_least_squares():
    """The fixed point is argmin ||P (A x - b)||, solved independently as a
    dense least-squares problem with P^T P = L L^T (Cholesky of the cropped
    circulant); the BB iterates reach it to 1e-9."""
    g = oracle.Geometry(8, 8, 8, 16)
    A = oracle.build_matrix(g)
    AT = A.transpose()
    b = np.random.default_rng(1).random((2, A.rows))
    x, _ = oracle.sirt_bb(A, AT, 8, b, 1000)
    Ad = scipy.sparse.csr_matrix((A.val, A.col, A.row_ptr), shape=(A.rows, A.cols)).toarray()
    hN = np.fft.ifft(oracle.ramp_response(8)).real
    N = hN.shape[0]
    T = np.array([[hN[(k - j) % N] for j in range(8)] for k in range(8)])
    L = np.linalg.cholesky(np.kron(np.eye(16), T))
    for s in range(2):
        ref = np.linalg.lstsq(L.T @ Ad, L.T @ b[s], rcond=None)[0]
        assert np.linalg.norm(x[s] - ref) <= 1e-9 * np.linalg.norm(ref)


def test_bb_step_is_exact_for_a_scaled_identity_hessian():
    """On f(x) = c/2 ||x - x*||^2 the BB1 step is 1/c, so the second step lands
    on x* exactly (Barzilai & Borwein, 1988).  Here A is the identity-like
    theta = 0 projector of a 1-pixel-high image (each ray meets one pixel with
    a unit chord) and the filter acts on single-bin rows, so the Hessian is
    D_eff * I with one scalar D_eff."""
    g = oracle.Geometry(1, 1, 1, 1)
    A = oracle.build_matrix(g)
    AT = A.transpose()
    assert A.nnz == 1 and A.val[0] == 1.0
    b = np.array([[3.0]])
    x, hist = oracle.sirt_bb(A, AT, 1, b, 3, first_step=0.7)
    assert x[0, 0] == pytest.approx(3.0, rel=1e-14)
    assert hist[2, 0] == pytest.approx(0.0, abs=1e-13)


def test_bb_resume_continues_the_same_iteration():
    g = oracle.Geometry(16, 16, 16, 20)
    A = oracle.build_matrix(g)
    AT = A.transpose()
    b = np.random.default_rng(4).random((3, A.rows))
    x_all, h_all = oracle.sirt_bb(A, AT, 16, b, 9)
    x, gp, a, fr, h1 = oracle.sirt_bb_resume(A, AT, 16, b, np.zeros((3, A.cols)), None, None, None, 4)
    x, gp, a, fr, h2 = oracle.sirt_bb_resume(A, AT, 16, b, x, gp, a, fr, 5)
    np.testing.assert_array_equal(x, x_all)
    np.testing.assert_array_equal(np.vstack([h1, h2]), h_all)


def test_bb_zero_data_freezes():
    g = oracle.Geometry(8, 8, 8, 6)
    A = oracle.build_matrix(g)
    x, hist = oracle.sirt_bb(A, A.transpose(), 8, np.zeros((1, A.rows)), 4)
    assert np.all(x == 0) and np.all(hist == 0)


# ---------------------------------------------------------------------------
# strip model: the area of the pixel square inside a unit-width strip
# ---------------------------------------------------------------------------

def clip_area(theta, p, xc, yc):
    """Area of the unit square centred (xc, yc) inside |x cos t + y sin t - p| <= 1/2:
    Sutherland-Hodgman clipping of the square against the two half-planes, then
    the shoelace formula."""
    c, s_ = math.cos(theta), math.sin(theta)
    poly = [(xc - 0.5, yc - 0.5), (xc + 0.5, yc - 0.5), (xc + 0.5, yc + 0.5), (xc - 0.5, yc + 0.5)]
    for sign, off in ((1.0, p + 0.5), (-1.0, -(p - 0.5))):   # sign*(x c + y s) <= off
        f = lambda q: sign * (q[0] * c + q[1] * s_) - off  # noqa: E731
        out = []
        for i in range(len(poly)):
            a, b = poly[i], poly[(i + 1) % len(poly)]
            fa, fb = f(a), f(b)
            if fa <= 0:
                out.append(a)
            if (fa < 0 < fb) or (fb < 0 < fa):
                t = fa / (fa - fb)
                out.append((a[0] + t * (b[0] - a[0]), a[1] + t * (b[1] - a[1])))
        poly = out
        if not poly:
            return 0.0
    area = 0.0
    for i in range(len(poly)):
        (x0, y0), (x1, y1) = poly[i], poly[(i + 1) % len(poly)]
        area += x0 * y1 - x1 * y0
    return abs(area) / 2


@pytest.mark.parametrize("nx,ny,n_p,center,angles", [
    (8, 8, 8, None, [0.0, math.pi / 4, math.pi / 2, 0.3, 1.1, 2.0, 2.9, 3.0]),
    (8, 8, 11, 5.3, [0.05, 0.7, 1.5707, 1.6, 2.356194490192345, 3.1]),
    (7, 9, 12, None, list(np.random.default_rng(3).uniform(0, math.pi, 10))),
])
def test_strip_weights_match_polygon_clipping(nx, ny, n_p, center, angles):
    g = oracle.Geometry(nx, ny, n_p, len(angles), np.array(angles), center, model="strip")
    c = g.c()
    for m, th in enumerate(angles):
        for k in range(n_p):
            p = k + 0.5 - c
            for iy in range(ny):
                for ix in range(nx):
                    ref = clip_area(th, p, ix + 0.5 - nx / 2, iy + 0.5 - ny / 2)
                    w = oracle.weight(g, m, k, ix, iy)
                    if w is None:
                        assert ref < 1e-12, (m, k, ix, iy, ref)
                    else:
                        assert abs(w - ref) < 1e-12, (m, k, ix, iy, w, ref)


def test_strip_mass_is_exact_per_angle():
    """Each pixel's weights over the bins of one angle add up to its area, 1,
    whenever its projection lies inside the detector (the strips tile the
    detector line)."""
    g = oracle.Geometry(24, 20, 30, 17, center=14.6, model="strip")
    A = oracle.build_matrix(g)
    AT = A.transpose()
    cs, sn = g.trig()
    c = g.c()
    checked = 0
    for j in range(A.cols):
        ix, iy = j % g.nx, j // g.nx
        x, y = ix + 0.5 - g.nx / 2, iy + 0.5 - g.ny / 2
        lo, hi = AT.row_ptr[j], AT.row_ptr[j + 1]
        rays, vals = AT.col[lo:hi], AT.val[lo:hi]
        for m in range(g.n_theta):
            a = max(abs(cs[m]), abs(sn[m]))
            e = min(abs(cs[m]), abs(sn[m]))
            t = x * cs[m] + y * sn[m]
            if t - 0.5 * (a + e) < -c or t + 0.5 * (a + e) > g.n_p - c:
                continue
            sel = (rays // g.n_p) == m
            assert abs(vals[sel].sum() - 1.0) < 1e-12
            checked += 1
    assert checked > 0.8 * A.cols * g.n_theta


def test_strip_theta_zero_is_column_sum():
    """theta = 0 with bins aligned to pixel columns: each pixel lies entirely
    in one strip (weight 1), so (A x)_k is the sum of image column k."""
    n = 9
    g = oracle.Geometry(n, n, n, 1, np.array([0.0]), model="strip")
    A = oracle.build_matrix(g)
    assert np.all(A.val == 1.0) and A.nnz == n * n
    x = np.random.default_rng(2).random((1, n * n))
    np.testing.assert_allclose(A.apply(x)[0], x.reshape(n, n).sum(axis=0), rtol=1e-15)

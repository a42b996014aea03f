"""Pins of the Fubini-Radon oracle (Sec. 3, Eq. 2) against facts that do not
come from its own code: the exact double sum (gridding error falling with the
window width), the analytic projection of a Gaussian blob, the real-space
projector of this build on smooth phantoms (Fourier-slice consistency), the
adjoint identity, the Kaiser-Bessel transform's closed form, and filtered
backprojection of analytic projections."""
import math

import numpy as np
import pytest

import oracle
from oracle import fubini as fb


def kb_hat_closed(s, kw, beta):
    """phi_hat(s) = kw sinh(sqrt(beta^2 - (pi kw s)^2)) / sqrt(beta^2 - (pi kw s)^2)
    (the Kaiser-Bessel window's transform, Jackson et al., IEEE TMI 1991)."""
    z = np.sqrt(beta ** 2 - (math.pi * kw * np.asarray(s)) ** 2)
    return kw * np.sinh(z) / z


@pytest.mark.parametrize("kw", [4, 6, 8])
def test_kb_quadrature_matches_closed_form(kw):
    beta = fb.kb_beta(kw)
    s = np.linspace(-0.25, 0.25, 11)
    np.testing.assert_allclose(fb.kb_hat(s, kw, beta), kb_hat_closed(s, kw, beta), rtol=1e-12)


def test_direct_is_the_gaussian_projection():
    """The exact transform of a sampled Gaussian blob (sigma 2.5 px, off
    centre, shifted axis) equals its continuous projection
    sqrt(2 pi) sigma exp(-(p - p0)^2 / (2 sigma^2)): the blob's spectrum vanishes
    beyond the sampled band."""
    n = 32
    fg = fb.FGeometry(n, n, 9, center=n / 2 - 0.3)
    sig, x0, y0 = 2.5, 1.3, -2.1
    c = fg.pix()
    X, Y = np.meshgrid(c, c)
    u = np.exp(-((X - x0) ** 2 + (Y - y0) ** 2) / (2 * sig ** 2)).ravel()[None]
    d = fb.fubini_direct(fg, u).reshape(9, n)
    p = fg.bins()
    ana = np.array([math.sqrt(2 * math.pi) * sig * np.exp(-(p - (x0 * math.cos(t) + y0 * math.sin(t))) ** 2
                                                        / (2 * sig ** 2)) for t in fg.theta()])
    assert np.abs(d - ana).max() <= 1e-6 * ana.max()


@pytest.mark.parametrize("kw,tol", [(4, 2e-3), (6, 2e-5), (8, 2e-7)])
def test_gridding_converges_to_the_direct_sum(kw, tol):
    """The gridded transform against the exact double sum on a random image
    supported in the inscribed disk: the error falls with the window width."""
    fg = fb.FGeometry(24, 26, 13, center=12.7, kw=kw)
    rng = np.random.default_rng(1)
    c = fg.pix()
    X, Y = np.meshgrid(c, c)
    u = rng.random((2, 24 * 24)) * ((X ** 2 + Y ** 2 < (0.45 * 24) ** 2).ravel())
    d = fb.fubini_direct(fg, u)
    assert np.linalg.norm(fb.fubini_project(fg, u) - d) <= tol * np.linalg.norm(d)


def test_adjoint_identity():
    fg = fb.FGeometry(24, 26, 13, center=12.7)
    S = fb.gridding_matrix(fg)
    rng = np.random.default_rng(2)
    u = rng.standard_normal((2, 24 * 24))
    y = rng.standard_normal((2, 13 * 26))
    lhs = np.sum(fb.fubini_project(fg, u, S) * y)
    rhs = np.sum(u * fb.fubini_backproject(fg, y, S))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_agrees_with_the_real_space_projector_on_a_smooth_phantom():
    """Fourier-slice consistency: on a Gaussian blob (sigma 4 px) the
    Fubini-Radon projections and the chord-length projector A of this build
    agree to the latter's discretisation error."""
    n, nt = 64, 30
    fg = fb.FGeometry(n, n, nt)
    g = oracle.Geometry(n, n, n, nt)
    A = oracle.build_matrix(g)
    c = fg.pix()
    X, Y = np.meshgrid(c, c)
    u = np.exp(-((X - 3.0) ** 2 + (Y + 5.0) ** 2) / (2 * 4.0 ** 2)).ravel()[None]
    rf = fb.fubini_project(fg, u)
    ra = A.apply(u)
    assert np.linalg.norm(rf - ra) <= 5e-3 * np.linalg.norm(ra)


def test_fbp_reconstructs_analytic_projections():
    """iRadon of the analytic projections of a centred Gaussian blob (sigma
    4 px) and of a uniform disk (radius 0.3 n): the blob within 3% (relative
    L2), the disk's interior level within 10%.  (The ramp sampled at the n_p
    radial points without padding leaves a small level error; a wrong scale
    factor would be off by far more.)"""
    n, nt = 128, 180
    fg = fb.FGeometry(n, n, nt)
    S = fb.gridding_matrix(fg)
    c = fg.pix()
    X, Y = np.meshgrid(c, c)
    p = fg.bins()
    sig = 4.0
    u = np.exp(-(X ** 2 + Y ** 2) / (2 * sig ** 2)).ravel()
    pg = np.tile(math.sqrt(2 * math.pi) * sig * np.exp(-p ** 2 / (2 * sig ** 2)), nt)[None]
    xg = fb.fubini_fbp(fg, pg, S)[0]
    assert np.linalg.norm(xg - u) <= 0.03 * np.linalg.norm(u)
    R = 0.3 * n
    pd = np.tile(np.where(np.abs(p) < R, 2 * np.sqrt(np.maximum(R * R - p * p, 0.0)), 0.0), nt)[None]
    xd = fb.fubini_fbp(fg, pd, S)[0].reshape(n, n)
    rr = np.sqrt(X ** 2 + Y ** 2)
    assert abs(xd[rr < 0.8 * R].mean() - 1.0) < 0.1


def test_hamming_density_ends():
    """The windowed density is the ramp density times 1 at DC and 0.08 at the
    Nyquist sample (q = 0, w = -1/2)."""
    fg = fb.FGeometry(16, 16, 4)
    r, h = fb.ramp_density(fg), fb.hamming_density(fg)
    assert h[fg.n_p // 2] == pytest.approx(r[fg.n_p // 2], rel=1e-15)
    assert h[0] == pytest.approx(0.08 * r[0], rel=1e-12)


def test_sirt_bb_first_step_is_the_fbp_and_it_solves_consistent_data():
    """The first iterate is the Hamming-filtered backprojection of b.  On
    consistent data b = R x_true of a smooth phantom (two Gaussian blobs), the
    iteration drives the residual to 1e-3 of its start and the iterate to
    x_true within 5e-3 in 30 steps (the FBP alone is 8% off): a descent
    method with the right gradient; a wrong sign or step rule diverges or
    stalls."""
    n, nt = 32, 40
    fg = fb.FGeometry(n, n, nt, kw=6)
    S = fb.gridding_matrix(fg)
    c = fg.pix()
    X, Y = np.meshgrid(c, c)
    xt = (np.exp(-((X - 3) ** 2 + (Y + 2) ** 2) / (2 * 3.0 ** 2))
          + 0.5 * np.exp(-((X + 5) ** 2 + (Y - 4) ** 2) / (2 * 2.0 ** 2))).ravel()[None]
    b = fb.fubini_project(fg, xt, S)
    x1, _ = fb.fubini_sirt_bb(fg, b, 1, S)
    np.testing.assert_allclose(x1, fb.fubini_fbp(fg, b, S, fb.hamming_density(fg)), rtol=1e-13, atol=1e-14)
    x, hist = fb.fubini_sirt_bb(fg, b, 30, S)
    assert hist[-1, 0] < 1e-3 * hist[0, 0]
    assert np.linalg.norm(x - xt) < 5e-3 * np.linalg.norm(xt)


# ---------------------------------------------------------------------------
# The normal operator N = R^T W R (Sec. 5's Toeplitz route): the exact
# backprojection, its agreement with the gridded one, the entry formula, and
# the SIRT that applies N in one step.

NORMAL_GEOMS = [
    dict(n=16, n_p=16, n_theta=12),                      # even n_p: a Hankel part
    dict(n=16, n_p=17, n_theta=10),                      # odd n_p: none
    dict(n=12, n_p=14, n_theta=9, center=6.3),           # off-centre axis
    dict(n=10, n_p=12, n_theta=7, angles=np.sort(np.random.default_rng(5).uniform(0, math.pi, 7))),
]


@pytest.mark.parametrize("g", range(len(NORMAL_GEOMS)))
def test_direct_backproject_is_the_exact_adjoint(g):
    fg = fb.FGeometry(**NORMAL_GEOMS[g])
    rng = np.random.default_rng(g)
    u = rng.standard_normal((2, fg.n * fg.n))
    y = rng.standard_normal((2, fg.n_theta * fg.n_p))
    lhs = np.sum(fb.fubini_direct(fg, u) * y)
    rhs = np.sum(u * fb.fubini_direct_backproject(fg, y, 0))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("filt", [0, 1, 2])
def test_direct_backproject_is_the_gridded_one_without_gridding_error(filt):
    """At kw = 8 the gridded adjoint / filtered backprojection (pinned on its
    own above) is within 3e-7 of the exact double sum."""
    fg = fb.FGeometry(24, 24, 20, kw=8)
    y = np.random.default_rng(filt).standard_normal((2, fg.n_theta * fg.n_p))
    ex = fb.fubini_direct_backproject(fg, y, filt)
    dens = [None, fb.ramp_density(fg), fb.hamming_density(fg)][filt]
    gr = fb.fubini_backproject(fg, y) if filt == 0 else fb.fubini_fbp(fg, y, None, dens)
    assert np.linalg.norm(ex - gr) <= 3e-7 * np.linalg.norm(ex)


@pytest.mark.parametrize("filt", [0, 1, 2])
def test_normal_is_symmetric_positive_semidefinite(filt):
    fg = fb.FGeometry(16, 16, 12)
    rng = np.random.default_rng(10 + filt)
    u, v = rng.standard_normal((2, 1, 256))
    Nu, Nv = fb.fubini_normal(fg, u, filt), fb.fubini_normal(fg, v, filt)
    assert abs(np.sum(Nu * v) - np.sum(u * Nv)) <= 1e-12 * np.linalg.norm(Nu) * np.linalg.norm(v)
    assert np.sum(Nu * u) > 0.0


@pytest.mark.parametrize("g", range(len(NORMAL_GEOMS)))
@pytest.mark.parametrize("filt", [0, 1, 2])
def test_normal_taps_are_its_entries(g, filt):
    """Columns N e_l of the composition against the Toeplitz + Hankel entry
    formula, every row j, three columns l."""
    fg = fb.FGeometry(**NORMAL_GEOMS[g])
    nn = fg.n * fg.n
    cols = [0, 5, nn // 2 + 3]
    Ncols = fb.fubini_normal(fg, np.eye(nn)[cols], filt)
    for r, l in enumerate(cols):
        d, s = fb.normal_entry_vectors(fg, np.arange(nn), np.full(nn, l))
        t, h = fb.normal_taps(fg, d, s, filt)
        assert np.abs(Ncols[r] - (t + h)).max() <= 1e-12 * np.abs(Ncols[r]).max()


@pytest.mark.parametrize("filt", [0, 1, 2])
def test_normal_is_the_gridded_composition_without_gridding_error(filt):
    fg = fb.FGeometry(32, 32, 24, kw=8)
    u = np.random.default_rng(20 + filt).standard_normal((2, 1024))
    ex = fb.fubini_normal(fg, u, filt)
    dens = [None, fb.ramp_density(fg), fb.hamming_density(fg)][filt]
    y = fb.fubini_project(fg, u)
    gr = fb.fubini_backproject(fg, y) if filt == 0 else fb.fubini_fbp(fg, y, None, dens)
    assert np.linalg.norm(ex - gr) <= 3e-7 * np.linalg.norm(ex)


def test_ramp_normal_is_near_identity_on_a_smooth_blob():
    """Filtered backprojection undoes the transform: N (ramp) leaves a
    Gaussian blob (sigma 4 px, n = 48, 80 angles) within 6% (the discrete
    ramp's DC weight and the angular sampling account for the rest)."""
    fg = fb.FGeometry(48, 48, 80)
    c = fg.pix()
    X, Y = np.meshgrid(c, c)
    u = np.exp(-(X ** 2 + Y ** 2) / (2 * 4.0 ** 2)).reshape(1, -1)
    assert np.linalg.norm(fb.fubini_normal(fg, u, 1) - u) <= 0.06 * np.linalg.norm(u)


def test_sirt_bb_normal_is_the_gridded_sirt_without_gridding_error():
    """The SIRT with N in one step: its first iterate is the Hamming-filtered
    backprojection of b, and at kw = 8 its 20-iteration trajectory is that of
    the SIRT that projects and backprojects every step (pinned above) within
    3e-7; the gradient norm falls below 1e-3 of its start."""
    n, nt = 32, 40
    fg = fb.FGeometry(n, n, nt, kw=8)
    S = fb.gridding_matrix(fg)
    c = fg.pix()
    X, Y = np.meshgrid(c, c)
    xt = (np.exp(-((X - 3) ** 2 + (Y + 2) ** 2) / (2 * 3.0 ** 2))
          + 0.5 * np.exp(-((X + 5) ** 2 + (Y - 4) ** 2) / (2 * 2.0 ** 2))).ravel()[None]
    b = fb.fubini_project(fg, xt, S)
    x1, _ = fb.fubini_sirt_bb_normal(fg, b, 1, S)
    np.testing.assert_allclose(x1, fb.fubini_fbp(fg, b, S, fb.hamming_density(fg)), rtol=1e-13, atol=1e-14)
    xn, hn = fb.fubini_sirt_bb_normal(fg, b, 20, S)
    xg, _ = fb.fubini_sirt_bb(fg, b, 20, S)
    assert np.linalg.norm(xn - xg) <= 3e-7 * np.linalg.norm(xg)
    assert hn[-1, 0] < 1e-3 * hn[0, 0]

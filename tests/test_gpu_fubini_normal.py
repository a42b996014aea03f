"""The normal operator of the Fubini-Radon transform in one step (the Toeplitz
route of Sec. 5) on the GPU vs the FP64 oracle, through the C ABI.

The oracle is the definition: the exact backprojection (adjoint, ramp or
Hamming iRadon) of the exact transform, as double sums.  The GPU applies it as
a circular convolution on the 2n x 2n grid with FP32 FFTs and spectra rounded
to FP32 once: 1e-5 relative L2 per slice (about eps32 log2(4 n^2) from the two
FFTs).  At the benchmark size, columns N e_l are checked entry by entry against
the oracle's entry formula, and the whole operator against the GPU's gridded
backprojection of its gridded projection (equal up to the gridding error)."""
import math

import numpy as np
import pytest

from oracle import fubini as fb
from paper_2003_12677_b300 import _lib, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # the gpu marker is only run on a GPU machine
    pytest.skip("needs CUDA", allow_module_level=True)

import paper_2003_12677_b300 as tomo  # noqa: E402


def per_slice_rel(a, b):
    a = np.asarray(a, np.float64).reshape(len(a), -1)
    b = np.asarray(b, np.float64).reshape(len(b), -1)
    return np.array([np.linalg.norm(a[i] - b[i]) / max(np.linalg.norm(b[i]), 1e-300) for i in range(len(a))])


_cache = {}


def pair(n, nt, n_p=None, center=None, angles=None, kw=6):
    key = (n, nt, n_p, center, None if angles is None else tuple(angles), kw)
    if key not in _cache:
        fg = fb.FGeometry(n, n if n_p is None else n_p, nt, None if angles is None else np.asarray(angles),
                          center, kw)
        F = tomo.Fubini(n, nt, n_p=n_p, angles=angles, center=center, kw=kw)
        _cache[key] = (fg, F)
    return _cache[key]


GEOS = [dict(n=16, nt=12),                                  # even n_p: Toeplitz + Hankel
        dict(n=16, nt=10, n_p=17),                          # odd n_p: Toeplitz only
        dict(n=12, nt=9, n_p=14, center=6.3),               # off-centre axis
        dict(n=10, nt=7, n_p=12, angles=[0.0, 0.4, 1.0, math.pi / 2, 2.2, 2.7, 3.0]),
        dict(n=40, nt=30)]


@pytest.mark.parametrize("geo", range(len(GEOS)))
@pytest.mark.parametrize("filt", [0, 1, 2])
def test_normal_matches_oracle(geo, filt):
    fg, F = pair(**GEOS[geo])
    for nz in (1, 3):
        x = inputs.random_slices((nz, fg.n, fg.n), 100 + geo * 7 + filt + nz)
        got = F.normal(torch.from_numpy(x).cuda(), [False, True, "hamming"][filt]).cpu().numpy()
        ref = fb.fubini_normal(fg, x.reshape(nz, -1), filt)
        assert per_slice_rel(got, ref).max() < 1e-5, (geo, filt, nz)


@pytest.mark.parametrize("n,nt", [(32, 24), (64, 30), (128, 40), (256, 12)])
def test_normal_fused_sizes_match_oracle(n, nt):
    """The 2n x 2n grid a power of two (64 .. 512 here): the fused convolution
    (register FFTs, no cuFFT); two slices per filter."""
    fg, F = pair(n=n, nt=nt)
    for filt in (0, 1, 2):
        x = inputs.random_slices((2, n, n), 150 + n + filt)
        got = F.normal(torch.from_numpy(x).cuda(), [False, True, "hamming"][filt]).cpu().numpy()
        ref = fb.fubini_normal(fg, x.reshape(2, -1), filt)
        assert per_slice_rel(got, ref).max() < 1e-5, (n, filt)


def test_normal_spans_passes():
    """More slices than one pass holds (32 for the cuFFT path at n = 12, 64 for
    the fused path at n = 16) and a ragged last pass; every slice equal to its
    single-slice result."""
    for n, nt, nz in ((12, 9, 33), (16, 12, 65)):
        fg, F = pair(n=n, nt=nt)
        x = inputs.random_slices((nz, n, n), 131 + n)
        got = F.normal(torch.from_numpy(x).cuda(), "hamming").cpu().numpy()
        ref = fb.fubini_normal(fg, x.reshape(nz, -1), 2)
        assert per_slice_rel(got, ref).max() < 1e-5
        one = F.normal(torch.from_numpy(x[nz - 1:]).cuda(), "hamming").cpu().numpy()
        np.testing.assert_array_equal(one[0], got[nz - 1])


def test_normal_full_size_columns_512x360():
    """512 x 512, 360 angles: N applied to four unit impulses (centre, corner,
    edge, interior), 64 sampled entries of each column vs the oracle's entry
    formula t(x_j - x_l) + h(x_j + x_l), within 1e-5 of the column's peak."""
    n, nt = 512, 360
    fg, F = pair(n=n, nt=nt)
    ls = [n * (n // 2) + n // 2, 0, n * 7 + n - 1, n * 300 + 123]
    e = np.zeros((4, n * n), np.float32)
    for i, l in enumerate(ls):
        e[i, l] = 1.0
    rng = np.random.default_rng(141)
    for filt in (0, 2):
        col = F.normal(torch.from_numpy(e.reshape(4, n, n)).cuda(), [False, True, "hamming"][filt])
        col = col.reshape(4, -1).cpu().numpy().astype(np.float64)
        for i, l in enumerate(ls):
            j = np.concatenate([[l, l + 1 if l + 1 < n * n else l - 1], rng.integers(0, n * n, 62)])
            d, s = fb.normal_entry_vectors(fg, j, np.full(j.shape, l))
            t, h = fb.normal_taps(fg, d, s, filt)
            peak = np.abs(col[i]).max()
            assert np.abs(col[i, j] - (t + h)).max() <= 1e-5 * peak, (filt, l)


def test_normal_is_the_gridded_composition_512x360():
    """At any size N x equals backproject(project(x)) of the gridded transform
    up to the gridding error (about 1e-5 at kw = 6 in the oracle)."""
    fg, F = pair(n=512, nt=360)
    case = inputs.workload_case("sirt_512x360_b64", slices=[0, 1, 2])
    x = torch.from_numpy(case.phantom).cuda()
    for filt in (0, 1, 2):
        f = [False, True, "hamming"][filt]
        got = F.normal(x, f).cpu().numpy()
        ref = F.backproject(F.project(x), f).cpu().numpy()
        assert per_slice_rel(got, ref).max() < 1e-4, filt


@pytest.mark.parametrize("geo", [dict(n=32, nt=40), dict(n=24, nt=20, n_p=25, center=12.2)])
def test_sirt_bb_normal_matches_oracle(geo):
    """The SIRT with N in one step: the first iterate is the GPU's gridded
    Hamming iRadon of b (1e-6), and 10 iterations track the FP64 oracle within
    1e-4, the gradient-norm history too."""
    fg, F = pair(**geo)
    if fg.n_p == fg.n:
        sino = inputs.make_case(fg.n, fg.n_theta, 3, seed=801, phantom="ellipses2d", noise="poisson",
                                level=1e5).sino
    else:  # no phantom generator for n_p != n: plain seeded data
        sino = inputs.random_slices((3, fg.n_theta, fg.n_p), 802)
    b = torch.from_numpy(sino).cuda()
    x1 = F.sirt_bb_normal(b, 1).cpu().numpy()
    np.testing.assert_array_less(per_slice_rel(x1, F.backproject(b, filtered="hamming").cpu().numpy()), 1e-6)
    x, h = F.sirt_bb_normal(b, 10, history=True)
    ref, href = fb.fubini_sirt_bb_normal(fg, sino.reshape(3, -1), 10)
    assert per_slice_rel(x.cpu().numpy(), ref).max() < 1e-4
    np.testing.assert_allclose(h.cpu().numpy(), href, rtol=1e-4)


@pytest.mark.parametrize("n,nt,nz", [(12, 9, 33), (16, 12, 65)])
def test_sirt_bb_normal_spans_passes_and_zero_iterations(n, nt, nz):
    """The cuFFT path (n = 12) over two passes of 32 and the fused path (n =
    16) over two passes of 64; 0 and 1 iterations."""
    fg, F = pair(n=n, nt=nt)
    c = inputs.make_case(n, nt, nz, seed=811, phantom="ellipses2d", noise="poisson", level=1e5)
    b = torch.from_numpy(c.sino).cuda()
    x, h = F.sirt_bb_normal(b, 6, history=True)
    ref, href = fb.fubini_sirt_bb_normal(fg, c.sino.reshape(nz, -1), 6)
    assert per_slice_rel(x.cpu().numpy(), ref).max() < 1e-4
    np.testing.assert_allclose(h.cpu().numpy(), href, rtol=1e-4)
    x0 = F.sirt_bb_normal(b[:2], 0)
    assert torch.count_nonzero(x0).item() == 0
    x1 = F.sirt_bb_normal(b[:2], 1).cpu().numpy()
    np.testing.assert_array_less(per_slice_rel(x1, F.backproject(b[:2], filtered="hamming").cpu().numpy()), 1e-6)


def test_sirt_bb_normal_tracks_the_gridded_sirt():
    """Both SIRTs on the same data (64 x 64, 90 angles): the iterates agree to
    the gridding error and FP32 rounding carried through 10 BB steps."""
    fg, F = pair(n=64, nt=90)
    c = inputs.make_case(64, 90, 4, seed=821, phantom="ellipses2d", noise="poisson", level=1e5)
    b = torch.from_numpy(c.sino).cuda()
    xn = F.sirt_bb_normal(b, 10).cpu().numpy()
    xg = F.sirt_bb(b, 10).cpu().numpy()
    assert per_slice_rel(xn, xg).max() < 1e-3


def test_normal_rejects_bad_arguments():
    fg, F = pair(n=16, nt=12)
    x = torch.zeros((1, 16, 16), device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(_lib.TomoError):
        _lib.call("tomo_fubini_normal", F._h, x.data_ptr(), y.data_ptr(), 1, 3, None)
    with pytest.raises(_lib.TomoError):
        _lib.call("tomo_fubini_normal", F._h, x.data_ptr(), y.data_ptr(), 0, 1, None)


@pytest.mark.parametrize("n,n_p,nt", [(1, 1, 1), (2, 3, 2), (3, 2, 5), (1, 4, 3)])
def test_degenerate_geometries(n, n_p, nt):
    """One-pixel images, one bin, one angle: the transform, its adjoint and the
    normal operator (cuFFT path, L = 2n < 32) against the oracle."""
    fg, F = pair(n=n, nt=nt, n_p=n_p)
    x = inputs.random_slices((2, n, n), 160 + n)
    y = inputs.random_slices((2, nt, n_p), 161 + n)
    gy = F.project(torch.from_numpy(x).cuda()).cpu().numpy()
    assert per_slice_rel(gy, fb.fubini_project(fg, x.reshape(2, -1))).max() < 1e-5
    gb = F.backproject(torch.from_numpy(y).cuda()).cpu().numpy()
    assert per_slice_rel(gb, fb.fubini_backproject(fg, y.reshape(2, -1))).max() < 1e-5
    for filt in (0, 1, 2):
        got = F.normal(torch.from_numpy(x).cuda(), [False, True, "hamming"][filt]).cpu().numpy()
        assert per_slice_rel(got, fb.fubini_normal(fg, x.reshape(2, -1), filt)).max() < 1e-5, filt


def test_normal_fused_2048_columns():
    """1024 x 1024 (2n = 2048: 64-point register DFTs, one block per SM):
    columns N e_l at three impulses against the oracle's entry formula (48
    sampled entries each, 1e-5 of the peak), and N against the gridded
    composition."""
    n, nt = 1024, 60
    fg, F = pair(n=n, nt=nt)
    ls = [n * (n // 2) + n // 2, 5, n * 900 + 1000]
    e = np.zeros((3, n * n), np.float32)
    for i, l in enumerate(ls):
        e[i, l] = 1.0
    rng = np.random.default_rng(171)
    for filt in (0, 2):
        col = F.normal(torch.from_numpy(e.reshape(3, n, n)).cuda(), [False, True, "hamming"][filt])
        col = col.reshape(3, -1).cpu().numpy().astype(np.float64)
        for i, l in enumerate(ls):
            j = np.concatenate([[l], rng.integers(0, n * n, 47)])
            d, s = fb.normal_entry_vectors(fg, j, np.full(j.shape, l))
            t, h = fb.normal_taps(fg, d, s, filt)
            assert np.abs(col[i, j] - (t + h)).max() <= 1e-5 * np.abs(col[i]).max(), (filt, l)
    x = torch.from_numpy(inputs.random_slices((2, n, n), 172)).cuda()
    got = F.normal(x, "hamming").cpu().numpy()
    ref = F.backproject(F.project(x), "hamming").cpu().numpy()
    assert per_slice_rel(got, ref).max() < 1e-4


def test_both_sirts_are_deterministic():
    """Fixed-order sums everywhere (BB sums, the long rows of S^T, the row-pair
    partials): two runs give the same bits, for the gridded SIRT and the SIRT
    with N."""
    fg, F = pair(n=64, nt=90)
    c = inputs.make_case(64, 90, 5, seed=831, phantom="ellipses2d", noise="poisson", level=1e5)
    b = torch.from_numpy(c.sino).cuda()
    for run in (lambda: F.sirt_bb(b, 8, history=True), lambda: F.sirt_bb_normal(b, 8, history=True)):
        x1, h1 = run()
        x2, h2 = run()
        assert torch.equal(x1, x2) and torch.equal(h1, h2)

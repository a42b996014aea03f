"""The Fubini-Radon transform (Sec. 3, Eq. 2) on the GPU vs the FP64 oracle,
through the C ABI.  The GPU runs the same gridding algorithm in FP32 (cuFFT
single precision, FP32 SpMM): forward, exact adjoint and filtered
backprojection within 1e-5 relative L2 per slice of the oracle's gridded
FP64 results (the FP32 FFTs of a 2n x 2n grid carry about eps32 log2(4 n^2)
relative error); the adjoint identity holds to 1e-5; and against the exact
double-sum definition the error is the gridding error plus the same FP32
term."""
import math

import numpy as np
import pytest

import oracle
from oracle import fubini as fb
from paper_2003_12677_b300 import inputs

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
        _cache[key] = (fg, fb.gridding_matrix(fg), F)
    return _cache[key]


GEOS = [dict(n=24, nt=13, n_p=26, center=12.7), dict(n=128, nt=180), dict(n=64, nt=30, kw=8),
        dict(n=40, nt=7, angles=[0.0, 0.3, 1.1, math.pi / 2, 2.0, 2.9, 3.1]),
        dict(n=40, nt=11, n_p=64, center=30.2)]  # radial register FFTs (n_p = 64) beside a cuFFT grid (G = 80)


@pytest.mark.parametrize("geo", GEOS)
@pytest.mark.parametrize("nz", [1, 5, 17])
def test_forward_adjoint_fbp_match_oracle(geo, nz):
    fg, S, F = pair(**geo)
    x = inputs.random_slices((nz, fg.n, fg.n), 21)
    y = inputs.random_slices((nz, fg.n_theta, fg.n_p), 22)
    gy = F.project(torch.from_numpy(x).cuda()).cpu().numpy()
    assert per_slice_rel(gy, fb.fubini_project(fg, x.reshape(nz, -1), S)).max() < 1e-5
    gx = F.backproject(torch.from_numpy(y).cuda()).cpu().numpy()
    assert per_slice_rel(gx, fb.fubini_backproject(fg, y.reshape(nz, -1), S)).max() < 1e-5
    gf = F.backproject(torch.from_numpy(y).cuda(), filtered=True).cpu().numpy()
    assert per_slice_rel(gf, fb.fubini_fbp(fg, y.reshape(nz, -1), S)).max() < 1e-5


def test_adjoint_identity_fp32():
    fg, S, F = pair(n=128, nt=180)
    xr = torch.from_numpy(inputs.random_slices((3, 128, 128), 31)).cuda()
    yr = torch.from_numpy(inputs.random_slices((3, 180, 128), 32)).cuda()
    lhs = torch.sum(F.project(xr).double() * yr.double()).item()
    rhs = torch.sum(xr.double() * F.backproject(yr).double()).item()
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_matches_the_exact_transform():
    """Against the double-sum definition: within the kw = 6 gridding error
    (3e-6, measured in the oracle) plus the FP32 term."""
    fg, S, F = pair(n=24, nt=13, n_p=26, center=12.7)
    c = fg.pix()
    X, Y = np.meshgrid(c, c)
    x = (inputs.random_slices((2, 24, 24), 41) * (X ** 2 + Y ** 2 < (0.45 * 24) ** 2)).astype(np.float32)
    gy = F.project(torch.from_numpy(x).cuda()).cpu().numpy()
    assert per_slice_rel(gy, fb.fubini_direct(fg, x.reshape(2, -1))).max() < 2e-5


def test_full_size_512x360():
    """The benchmark geometry: 512x512, 360 angles, 512 bins; 20 slices (two
    passes of 16) forward and filtered backprojection, two slices vs the oracle."""
    fg = fb.FGeometry(512, 512, 360)
    S = fb.gridding_matrix(fg)
    F = tomo.Fubini(512, 360)
    case = inputs.workload_case("sirt_512x360_b64", slices=list(range(20)))
    y = F.project(torch.from_numpy(case.phantom).cuda()).cpu().numpy()
    pick = [0, 17]
    assert per_slice_rel(y[pick], fb.fubini_project(fg, case.phantom[pick].reshape(2, -1), S)).max() < 1e-5
    xf = F.backproject(torch.from_numpy(case.sino).cuda(), filtered=True).cpu().numpy()
    assert per_slice_rel(xf[pick], fb.fubini_fbp(fg, case.sino[pick].reshape(2, -1), S)).max() < 1e-5
    F.close()


def test_hamming_fbp_matches_oracle():
    fg, S, F = pair(n=128, nt=180)
    y = inputs.random_slices((3, 180, 128), 51)
    gf = F.backproject(torch.from_numpy(y).cuda(), filtered="hamming").cpu().numpy()
    ref = fb.fubini_fbp(fg, y.reshape(3, -1), S, fb.hamming_density(fg))
    assert per_slice_rel(gf, ref).max() < 1e-5


def test_sirt_bb_matches_oracle():
    """The paper's SIRT on the Fubini-Radon operator: the first step is the
    Hamming-filtered backprojection (1e-5); 10 iterations track the FP64
    oracle within 1e-4 (the BB recurrence in FP32, as for the line model)."""
    fg, S, F = pair(n=64, nt=30, kw=8)
    c = inputs.make_case(64, 30, 3, seed=701, phantom="ellipses2d", noise="poisson", level=1e5)
    b = torch.from_numpy(c.sino).cuda()
    x1 = F.sirt_bb(b, 1).cpu().numpy()
    np.testing.assert_array_less(per_slice_rel(x1, F.backproject(b, filtered="hamming").cpu().numpy()), 1e-6)
    x, h = F.sirt_bb(b, 10, history=True)
    ref, href = fb.fubini_sirt_bb(fg, c.sino.reshape(3, -1), 10, S)
    assert per_slice_rel(x.cpu().numpy(), ref).max() < 1e-4
    np.testing.assert_allclose(h.cpu().numpy(), href, rtol=1e-4)


@pytest.mark.parametrize("n,nt", [(16, 12), (32, 20), (256, 40), (1024, 30)])
def test_register_fft_grids_match_oracle(n, nt):
    """Every power-of-two grid split of the register-FFT passes (G = 2n = 32 ..
    2048) and, with n_p = n, the radial ones (n_p = 32 .. 1024; 16 takes
    cuFFT): forward, adjoint and the Hamming iRadon against the oracle."""
    fg, S, F = pair(n=n, nt=nt)
    x = inputs.random_slices((3, n, n), 60 + n)
    y = inputs.random_slices((3, nt, n), 61 + n)
    gy = F.project(torch.from_numpy(x).cuda()).cpu().numpy()
    assert per_slice_rel(gy, fb.fubini_project(fg, x.reshape(3, -1), S)).max() < 1e-5
    gx = F.backproject(torch.from_numpy(y).cuda()).cpu().numpy()
    assert per_slice_rel(gx, fb.fubini_backproject(fg, y.reshape(3, -1), S)).max() < 1e-5
    gf = F.backproject(torch.from_numpy(y).cuda(), filtered="hamming").cpu().numpy()
    assert per_slice_rel(gf, fb.fubini_fbp(fg, y.reshape(3, -1), S, fb.hamming_density(fg))).max() < 1e-5

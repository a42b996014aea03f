"""The strip model (area of each pixel inside the unit-width strip of a bin)
on the GPU vs the FP64 oracle, through the C ABI: the same bars as the line
model -- structure bit-exact, FP32 values equal to the oracle's FP64 weights
rounded to nearest, FP32 SpMM within 1e-5, 16-bit SpMM within 5e-3 (bf16) /
1e-3 (f16), SIRT within 1e-4."""
import math

import numpy as np
import pytest

import oracle
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


def pair(nx, nt, n_p=None, ny=None, angles=None, center=None, values="f32"):
    key = (nx, nt, n_p, ny, None if angles is None else tuple(angles), center, values)
    if key not in _cache:
        g = oracle.Geometry(nx, nx if ny is None else ny, nx if n_p is None else n_p, nt,
                            None if angles is None else np.asarray(angles), center, model="strip")
        A = oracle.build_matrix(g)
        M = tomo.Matrix(nx, nt, n_p=n_p, n_y=ny, angles=angles, center=center, values=values, model="strip")
        _cache[key] = (g, A, A.transpose(), M)
    return _cache[key]


GEOMS = [
    dict(nx=128, nt=180),
    dict(nx=37, nt=23, n_p=41, center=19.7),
    dict(nx=40, nt=7, ny=29, n_p=50),
    dict(nx=16, nt=6, angles=[0.0, math.pi / 4, math.pi / 2, 3 * math.pi / 4, 1e-9, math.pi - 1e-9]),
    dict(nx=1, nt=1),
]


@pytest.mark.parametrize("geo", GEOMS)
def test_structure_and_values_bitexact(geo):
    g, A, AT, M = pair(**geo)
    assert M.nnz == A.nnz
    for tr, ref in ((False, A), (True, AT)):
        rp, col, val = M.export_csr(transpose=tr)
        np.testing.assert_array_equal(rp, ref.row_ptr)
        np.testing.assert_array_equal(col, ref.col)
        np.testing.assert_array_equal(val, ref.val.astype(np.float32))
    R, C = M.export_norms()
    rs = np.bincount(np.repeat(np.arange(A.rows), np.diff(A.row_ptr)), weights=A.val, minlength=A.rows)
    np.testing.assert_allclose(R, np.where(rs > 0, 1.0 / np.where(rs > 0, rs, 1.0), 0.0), rtol=1e-6)
    cs = np.bincount(A.col, weights=A.val, minlength=A.cols)
    np.testing.assert_allclose(C, np.where(cs > 0, 1.0 / np.where(cs > 0, cs, 1.0), 0.0), rtol=1e-6)


@pytest.mark.parametrize("B,fmt", [(1, "csr"), (4, "sell"), (16, "sell"), (64, "csr")])
def test_project_backproject(B, fmt):
    g, A, AT, M = pair(nx=128, nt=180)
    x = inputs.random_slices((5, 128, 128), 11)
    y = inputs.random_slices((5, 180, 128), 12)
    px = tomo.project(M, torch.from_numpy(x).cuda(), batch_width=B, fmt=fmt).cpu().numpy()
    by = tomo.backproject(M, torch.from_numpy(y).cuda(), batch_width=B, fmt=fmt).cpu().numpy()
    assert per_slice_rel(px, A.apply(x.reshape(5, -1))).max() < 1e-5
    assert per_slice_rel(by, AT.apply(y.reshape(5, -1))).max() < 1e-5


@pytest.mark.parametrize("values,tol", [("bf16", 5e-3), ("f16", 1e-3)])
def test_16bit_spmm(values, tol):
    g, A, AT, M = pair(nx=128, nt=180, values=values)
    x = inputs.random_slices((4, 128, 128), 13)
    px = tomo.project(M, torch.from_numpy(x).cuda(), batch_width=4, fmt="sell16").cpu().numpy()
    assert per_slice_rel(px, A.apply(x.reshape(4, -1))).max() < tol
    y = inputs.random_slices((4, 180, 128), 14)
    by = tomo.backproject(M, torch.from_numpy(y).cuda(), batch_width=4, fmt="sell16").cpu().numpy()
    assert per_slice_rel(by, AT.apply(y.reshape(4, -1))).max() < tol


@pytest.mark.parametrize("B", [1, 8])
def test_sirt_50(B):
    g, A, AT, M = pair(nx=128, nt=180)
    c = inputs.make_case(128, 180, 3, seed=601, phantom="ellipses2d", noise="poisson", level=1e5)
    x = tomo.sirt(M, torch.from_numpy(c.sino).cuda(), 50, batch_width=B).cpu().numpy()
    ref = oracle.sirt(A, AT, c.sino.reshape(3, -1), 50)
    assert per_slice_rel(x, ref).max() < 1e-4


def test_full_size_sampled_rows_512x360():
    """512x512 pixels, 360 angles: sampled rows of A and A^T bit-exact against
    the oracle's brute-force rows; the total entry count equals the oracle's."""
    g = oracle.Geometry(512, 512, 512, 360, model="strip")
    M = tomo.Matrix(512, 360, model="strip")
    for i in [0, 511, 180 * 512 + 256, 90 * 512 + 3, 359 * 512 + 500, 45 * 512 + 300]:
        rp, col, val = M.export_rows(i, i + 1)
        c2, v2 = oracle.row(g, i)
        np.testing.assert_array_equal(col, c2)
        np.testing.assert_array_equal(val, v2.astype(np.float32))
    for j in [0, 511, 256 * 512 + 256, 512 * 512 - 1, 100 * 512 + 7]:
        rp, col, val = M.export_rows(j, j + 1, transpose=True)
        c2, v2 = oracle.pixel_row(g, j)
        np.testing.assert_array_equal(col, c2)
        np.testing.assert_array_equal(val, v2.astype(np.float32))
    A = oracle.build_matrix(g)
    assert M.nnz == A.nnz
    M.close()

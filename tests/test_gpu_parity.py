"""CUDA path vs the FP64 oracle, through the C ABI (ctypes binding).

Bars: row pointers and column indices bit-exact; FP32 values equal to the
oracle's FP64 chord lengths rounded to nearest; FP32 SpMM within 1e-5
relative L2 per slice; SIRT and CGLS iterates within 1e-4 relative L2;
16-bit SpMM within 5e-3 (bf16) / 1e-3 (f16).
"""
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
from paper_2003_12677_b300 import _lib  # noqa: E402

WIDTHS = [1, 2, 4, 8, 16, 32, 64]


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def per_slice_rel(a, b):
    a = np.asarray(a, np.float64).reshape(len(a), -1)
    b = np.asarray(b, np.float64).reshape(len(b), -1)
    return np.array([rel_l2(a[i], b[i]) for i in range(len(a))])


_cache = {}


def pair(nx, nt, n_p=None, ny=None, angles=None, center=None, values="f32"):
    """(oracle geometry, oracle A, oracle A^T, GPU matrix) for one geometry."""
    key = (nx, nt, n_p, ny, None if angles is None else tuple(angles), center, values)
    if key not in _cache:
        g = oracle.Geometry(nx, nx if ny is None else ny, nx if n_p is None else n_p, nt,
                            None if angles is None else np.asarray(angles), center)
        A = oracle.build_matrix(g)
        M = tomo.Matrix(nx, nt, n_p=n_p, n_y=ny, angles=angles, center=center, values=values)
        _cache[key] = (g, A, A.transpose(), M)
    return _cache[key]


GEOMS = [
    dict(nx=128, nt=180),                                   # the 128x128, 180-angle workload
    dict(nx=37, nt=23, n_p=41, center=19.7),                # odd sizes, shifted axis
    dict(nx=40, nt=7, ny=29, n_p=50),                       # rectangular image, wide detector
    dict(nx=16, nt=6, angles=[0.0, math.pi / 4, math.pi / 2, 3 * math.pi / 4, 1e-9, math.pi - 1e-9]),
    dict(nx=1, nt=1),                                       # one pixel, one ray
]


@pytest.mark.parametrize("geo", GEOMS)
def test_structure_and_values_bitexact(geo):
    g, A, AT, M = pair(**geo)
    assert M.nnz == A.nnz
    rp, col, val = M.export_csr()
    np.testing.assert_array_equal(rp, A.row_ptr)
    np.testing.assert_array_equal(col, A.col)
    np.testing.assert_array_equal(val, A.val.astype(np.float32))
    rp, col, val = M.export_csr(transpose=True)
    np.testing.assert_array_equal(rp, AT.row_ptr)
    np.testing.assert_array_equal(col, AT.col)
    np.testing.assert_array_equal(val, AT.val.astype(np.float32))


@pytest.mark.parametrize("geo", GEOMS[:3])
def test_sirt_normalisers(geo):
    g, A, AT, M = pair(**geo)
    R, C = M.export_norms()
    np.testing.assert_allclose(R, oracle.inv_row_sums(A).astype(np.float32), rtol=2e-7, atol=0)
    np.testing.assert_allclose(C, oracle.inv_row_sums(AT).astype(np.float32), rtol=2e-7, atol=0)


@pytest.mark.parametrize("fmt", ["sell", "csr"])
@pytest.mark.parametrize("B", WIDTHS)
@pytest.mark.parametrize("nz", [1, 3, 9])
def test_project_backproject_f32(B, nz, fmt):
    g, A, AT, M = pair(nx=96, nt=60, n_p=101, center=50.3)
    x = inputs.random_slices((nz, 96, 96), seed=100 + nz)
    y = inputs.random_slices((nz, 60, 101), seed=200 + nz)
    yd = tomo.project(M, torch.from_numpy(x).cuda(), batch_width=B, fmt=fmt).cpu().numpy()
    xd = tomo.backproject(M, torch.from_numpy(y).cuda(), batch_width=B, fmt=fmt).cpu().numpy()
    assert per_slice_rel(yd, A.apply(x)).max() < 1e-5
    assert per_slice_rel(xd, AT.apply(y)).max() < 1e-5


@pytest.mark.parametrize("B", WIDTHS)
def test_interleaved_layout(B):
    g, A, AT, M = pair(nx=64, nt=45)
    x = inputs.random_slices((B, 64 * 64), seed=7)
    xi = torch.from_numpy(np.ascontiguousarray(x.T)).cuda()
    yi = tomo.project(M, xi, interleaved=True).cpu().numpy()
    assert per_slice_rel(yi.T, A.apply(x)).max() < 1e-5
    xb = tomo.backproject(M, torch.from_numpy(np.ascontiguousarray(yi)).cuda(), interleaved=True).cpu().numpy()
    assert per_slice_rel(xb.T, AT.apply(yi.T)).max() < 1e-5


def test_adjoint_identity_f32():
    g, A, AT, M = pair(nx=128, nt=180)
    x = torch.from_numpy(inputs.random_slices((4, 128, 128), 1)).cuda()
    y = torch.from_numpy(inputs.random_slices((4, 180, 128), 2)).cuda()
    lhs = torch.sum(tomo.project(M, x).double() * y.double()).item()
    rhs = torch.sum(x.double() * tomo.backproject(M, y).double()).item()
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


@pytest.mark.parametrize("fmt", ["sell", "csr"])
@pytest.mark.parametrize("B", [1, 4, 16])
def test_sirt_128(B, fmt):
    """one 128x128 slice, 180 angles, Poisson 1e5, SIRT 50 (and a 3-slice batch)."""
    c = inputs.workload_case("sirt_128x180_b1")
    g, A, AT, M = pair(nx=128, nt=180)
    sino = np.concatenate([c.sino, c.sino * 0.5, c.sino[:, ::-1]]) if B > 1 else c.sino
    sino = np.ascontiguousarray(sino)
    ref = oracle.sirt(A, AT, sino.reshape(len(sino), -1), 50, 1.0)
    got = tomo.sirt(M, torch.from_numpy(sino).cuda(), 50, batch_width=B, fmt=fmt).cpu().numpy()
    assert per_slice_rel(got, ref).max() < 1e-4


def test_sirt_lambda_and_start():
    g, A, AT, M = pair(nx=37, nt=23, n_p=41, center=19.7)
    rng = np.random.default_rng(3)
    b = rng.random((2, A.rows)).astype(np.float32)
    x0 = rng.random((2, 37 * 37)).astype(np.float32)
    ref = oracle.sirt(A, AT, b, 20, 0.7, x0=x0)
    got = tomo.sirt(M, torch.from_numpy(b).cuda(), 20, lam=0.7,
                    x0=torch.from_numpy(x0.reshape(2, 37, 37)).cuda(), batch_width=2).cpu().numpy()
    assert per_slice_rel(got, ref).max() < 1e-4


@pytest.mark.parametrize("B,nz", [(1, 2), (4, 5), (16, 16), (64, 3)])
@pytest.mark.parametrize("graph", [True, False])
@pytest.mark.parametrize("fmt", ["sell", "csr"])
def test_cgls(B, nz, graph, fmt):
    g, A, AT, M = pair(nx=64, nt=90)
    c = inputs.make_case(64, 90, nz, seed=55, phantom="ellipsoids3d", noise="gaussian", level=0.05)
    ref, href = oracle.cgls(A, AT, c.sino.reshape(nz, -1), 4)
    got, h = tomo.cgls(M, torch.from_numpy(c.sino).cuda(), 4, history=True, batch_width=B, use_graph=graph,
                       fmt=fmt)
    assert per_slice_rel(got.cpu().numpy(), ref).max() < 1e-4
    np.testing.assert_allclose(h.cpu().numpy(), href, rtol=1e-4)


def test_cgls_residual_recompute():
    g, A, AT, M = pair(nx=64, nt=90)
    c = inputs.make_case(64, 90, 4, seed=56, phantom="ellipsoids3d", noise="gaussian", level=0.05)
    ref, _ = oracle.cgls(A, AT, c.sino.reshape(4, -1), 4)
    got = tomo.cgls(M, torch.from_numpy(c.sino).cuda(), 4, recompute_every=2, batch_width=4)
    assert per_slice_rel(got.cpu().numpy(), ref).max() < 1e-4


@pytest.mark.parametrize("B", [1, 4])
def test_cgls_checkpoint_resume_is_bitwise(B):
    """25 iterations + resume for 25 gives the bits of 50 iterations."""
    g, A, AT, M = pair(nx=64, nt=90)
    c = inputs.make_case(64, 90, 3, seed=57, phantom="ellipsoids3d", noise="gaussian", level=0.05)
    sino = torch.from_numpy(c.sino).cuda()
    x50, h50 = tomo.cgls(M, sino, 50, recompute_every=5, history=True, batch_width=B)
    x25, h25, st = tomo.cgls(M, sino, 25, recompute_every=5, history=True, batch_width=B, return_state=True)
    xr, hr = tomo.cgls(M, sino, 25, recompute_every=5, history=True, batch_width=B, resume=st)
    assert torch.equal(xr, x50)
    assert torch.equal(torch.cat([h25, hr]), h50)


@pytest.mark.parametrize("fmt,B", [("sell", 1), ("sell", 16), ("csr", 4)])
def test_cgls_every_step_matches_an_oracle_step(fmt, B):
    """Each of 50 GPU CGLS steps, taken from the GPU's own state, equals one
    FP64 oracle step from that state (relative L2 1e-5 on x, r, p; 1e-5 on
    gamma).  This checks every step of the 50-iteration recurrence without the
    divergence that FP32 rounding causes when whole trajectories are compared."""
    c = inputs.workload_case("sirt_128x180_b1")
    g, A, AT, M = pair(nx=128, nt=180)
    sino_np = np.concatenate([c.sino, c.sino[:, ::-1]])
    sino = torch.from_numpy(np.ascontiguousarray(sino_np)).cuda()
    x, st = tomo.cgls(M, sino, 0, batch_width=B, fmt=fmt, return_state=True)
    for k in range(50):
        x1, st1 = tomo.cgls(M, sino, 1, batch_width=B, fmt=fmt, resume=st, return_state=True)
        ref = oracle.cgls_resume(A, AT, st["x"].double().cpu().numpy(), st["r"].double().cpu().numpy(),
                                 st["p"].double().cpu().numpy(), st["gamma"].cpu().numpy(),
                                 st["frozen"].cpu().numpy(), 1)
        assert per_slice_rel(x1.cpu().numpy(), ref[0]).max() < 1e-5, k
        assert per_slice_rel(st1["r"].cpu().numpy(), ref[1]).max() < 1e-5, k
        assert per_slice_rel(st1["p"].cpu().numpy(), ref[2]).max() < 1e-5, k
        np.testing.assert_allclose(st1["gamma"].cpu().numpy(), ref[3], rtol=1e-5)
        st = st1


UNEVEN = [(64, 90, 1), (96, 120, 5), (64, 90, 3), (128, 180, 7), (96, 120, 2), (64, 90, 9), (128, 180, 1)]


def _uneven_case():
    reqs, refs = [], []
    for k, (n, nt, nz) in enumerate(UNEVEN):
        g, A, AT, M = pair(nx=n, nt=nt)
        c = inputs.make_case(n, nt, nz, seed=300 + k, phantom="ellipses2d", noise="poisson", level=1e5)
        reqs.append((M, torch.from_numpy(c.sino).cuda()))
        refs.append((A, AT, c.sino.reshape(nz, -1)))
    return reqs, refs


@pytest.mark.parametrize("B", [4, 16])
def test_cgls_batched_uneven_matches_oracle(B):
    """7 requests, 3 geometries, 1-9 slices each, one persistent launch: each
    slice matches the FP64 oracle at 1e-4 over the iterations FP32 CGLS tracks
    it (4); repeated launches are bit-identical; the residual norm never
    increases over 30 iterations."""
    reqs, refs = _uneven_case()
    xs, hs = tomo.cgls_batched(reqs, 4, batch_width=B, history=True)
    for x, h, (A, AT, b) in zip(xs, hs, refs):
        ref, href = oracle.cgls(A, AT, b, 4)
        assert per_slice_rel(x.cpu().numpy(), ref).max() < 1e-4
        np.testing.assert_allclose(h.cpu().numpy(), href, rtol=1e-4)
    xs, hs = tomo.cgls_batched(reqs, 30, batch_width=B, history=True)
    xs2, _ = tomo.cgls_batched(reqs, 30, batch_width=B, history=True)
    for x, x2, h in zip(xs, xs2, hs):
        assert torch.equal(x, x2)                       # deterministic reductions
        hh = h.cpu().numpy()
        assert np.all(np.diff(hh, axis=0) <= 1e-6 * hh[0])  # ||r|| never increases


def test_cgls_batched_every_step_matches_an_oracle_step():
    """30 single-iteration persistent launches, each resumed from the state the
    previous one returned: every step equals one FP64 oracle step from that
    state within 1e-5 (x, r, p, gamma), for every slice of every request."""
    reqs, refs = _uneven_case()
    _, st = tomo.cgls_batched(reqs, 0, batch_width=8, return_state=True)
    for k in range(30):
        xs, st1 = tomo.cgls_batched(reqs, 1, batch_width=8, resume=st, return_state=True)
        for i, (A, AT, b) in enumerate(refs):
            s = st[i]
            ref = oracle.cgls_resume(A, AT, s["x"].double().cpu().numpy(), s["r"].double().cpu().numpy(),
                                     s["p"].double().cpu().numpy(), s["gamma"].cpu().numpy(),
                                     s["frozen"].cpu().numpy(), 1)
            assert per_slice_rel(xs[i].cpu().numpy(), ref[0]).max() < 1e-5, (k, i)
            assert per_slice_rel(st1[i]["r"].cpu().numpy(), ref[1]).max() < 1e-5, (k, i)
            assert per_slice_rel(st1[i]["p"].cpu().numpy(), ref[2]).max() < 1e-5, (k, i)
            np.testing.assert_allclose(st1[i]["gamma"].cpu().numpy(), ref[3], rtol=1e-5)
        st = st1


@pytest.mark.parametrize("values", ["bf16", "f16"])
def test_cgls_batched_16bit(values):
    """The persistent batched CGLS on 16-bit values: 4 iterations within 1e-4
    of the FP64 oracle run on the same 16-bit values (the FP32 arithmetic's
    bar; the value rounding's effect on accuracy is measured at equal data fit
    in test_gpu_cgls_accuracy.py)."""
    reqs, refs = [], []
    for k, (n, nt, nz) in enumerate([(64, 90, 3), (96, 120, 2)]):
        g, A, AT, M = pair(nx=n, nt=nt, values=values)
        c = inputs.make_case(n, nt, nz, seed=400 + k, phantom="ellipses2d", noise="poisson", level=1e5)
        reqs.append((M, torch.from_numpy(c.sino).cuda()))
        refs.append((_oracle16(g, A, values), c.sino.reshape(nz, -1)))
    xs = tomo.cgls_batched(reqs, 4, batch_width=4, fmt="sell16")
    for x, ((A16, AT16), b) in zip(xs, refs):
        ref, _ = oracle.cgls(A16, AT16, b, 4)
        assert per_slice_rel(x.cpu().numpy(), ref).max() < 1e-4


def test_cgls_batched_barrier_timeout_is_reported():
    """One block never arrives at the first grid barrier: every other block
    waits out the 50 ms limit, the launch ends and the call reports
    TOMO_ERR_TIMEOUT; the context stays usable."""
    reqs, refs = _uneven_case()
    with pytest.raises(_lib.TomoError) as ei:
        tomo.cgls_batched(reqs[:2], 3, batch_width=4, timeout_s=0.05, test_flags=1)
    assert ei.value.code == 4
    xs = tomo.cgls_batched(reqs[:2], 2, batch_width=4)
    ref, _ = oracle.cgls(*refs[0][:2], refs[0][2], 2)
    assert per_slice_rel(xs[0].cpu().numpy(), ref).max() < 1e-4


def test_cgls_batched_async_status_word():
    """Asynchronous batched launches: the call returns once queued; the
    stream's status word then reads TOMO_OK for a normal launch (whose result
    equals the synchronous one bit for bit) and TOMO_ERR_TIMEOUT for a launch
    in which one block never arrives; reading the word resets it."""
    reqs, refs = _uneven_case()
    assert tomo.stream_status() == "TOMO_OK"
    ref_xs = tomo.cgls_batched(reqs[:3], 5, batch_width=8)
    xs = tomo.cgls_batched(reqs[:3], 5, batch_width=8, asynchronous=True)
    assert tomo.stream_status() == "TOMO_OK"
    for x, r in zip(xs, ref_xs):
        assert torch.equal(x, r)
    tomo.cgls_batched(reqs[:2], 3, batch_width=4, timeout_s=0.05, test_flags=1, asynchronous=True)
    assert tomo.stream_status() == "TOMO_ERR_TIMEOUT"
    assert tomo.stream_status() == "TOMO_OK"
    # a side stream keeps a word of its own
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        tomo.cgls_batched(reqs[:2], 3, batch_width=4, timeout_s=0.05, test_flags=1, asynchronous=True)
    assert tomo.stream_status() == "TOMO_OK"
    assert tomo.stream_status(side) == "TOMO_ERR_TIMEOUT"


def test_cgls_zero_sinogram_is_frozen():
    g, A, AT, M = pair(nx=64, nt=90)
    z = torch.zeros((3, 90, 64), device="cuda")
    x, h = tomo.cgls(M, z, 5, history=True, batch_width=4)
    assert torch.all(x == 0) and torch.all(h == 0)


@pytest.mark.parametrize("values,tol", [("bf16", 5e-3), ("f16", 1e-3)])
@pytest.mark.parametrize("B", [1, 2, 4, 16, 64])
def test_lowprec_spmm(values, tol, B):
    g, A, AT, M = pair(nx=128, nt=180, values=values)
    x = inputs.random_slices((5, 128, 128), seed=31)
    y = inputs.random_slices((5, 180, 128), seed=32)
    yd = tomo.project(M, torch.from_numpy(x).cuda(), batch_width=B, fmt="sell16").cpu().numpy()
    xd = tomo.backproject(M, torch.from_numpy(y).cuda(), batch_width=B, fmt="sell16").cpu().numpy()
    assert per_slice_rel(yd, A.apply(x)).max() < tol
    assert per_slice_rel(xd, AT.apply(y)).max() < tol


def test_autograd_matches_oracle_gradient():
    """loss = ||A x - b||^2 + mu TV_eps(x): GPU autograd gradient vs the FP64
    oracle gradient on 64 random directions (relative 1e-4)."""
    n, nt, nz = 64, 60, 2
    g, A, AT, M = pair(nx=n, nt=nt)
    rng = np.random.default_rng(12)
    x = rng.random((nz, n, n)).astype(np.float32)
    b = rng.random((nz, nt, n)).astype(np.float32)
    mu, eps = 1e-3, 1e-3
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    r = tomo.radon(xt, M) - torch.from_numpy(b).cuda()
    loss = (r * r).sum() + mu * tomo.tv_loss(xt, eps)
    loss.backward()
    gd = xt.grad.double().cpu().numpy().reshape(nz, -1)
    f, gref = oracle.loss_grad(A, AT, n, n, x.reshape(nz, -1), b.reshape(nz, -1), mu, eps)
    assert abs(loss.item() - f) <= 1e-5 * abs(f)
    for _ in range(64):
        v = rng.standard_normal(gd.shape)
        v /= np.linalg.norm(v)
        a, e = float(np.sum(gd * v)), float(np.sum(gref * v))
        assert abs(a - e) <= 1e-4 * np.linalg.norm(gref)


@pytest.mark.parametrize("values", ["bf16", "f16"])
def test_lowprec_corner_gaps(values):
    """Corner pixels at 256x256 / 720 angles are seen by two angle ranges ~90
    degrees apart, so consecutive entries of their A^T rows jump by more than
    65535 columns; the 16-bit encoder must cut segments there."""
    g, A, AT, M = pair(nx=256, nt=720, values=values)
    tol = 5e-3 if values == "bf16" else 1e-3
    x = inputs.random_slices((4, 256, 256), seed=41)
    y = inputs.random_slices((4, 720, 256), seed=42)
    yd = tomo.project(M, torch.from_numpy(x).cuda(), batch_width=4, fmt="sell16").cpu().numpy()
    xd = tomo.backproject(M, torch.from_numpy(y).cuda(), batch_width=4, fmt="sell16").cpu().numpy()
    assert per_slice_rel(yd, A.apply(x)).max() < tol
    assert per_slice_rel(xd, AT.apply(y)).max() < tol


def test_autotune_choice_is_used_by_default():
    """The tuner searches width x format x A^T row-group order, then fewer
    resident blocks per SM for the best shape; calls with the defaults use its
    choice and give the bits of the explicit choice; every order and block
    count gives the same bits (the order of rows changes no sum)."""
    g, A, AT, M = pair(nx=128, nt=180)
    res = M.autotune(6)
    assert res["batch_width"] in (1, 2, 4, 8) and res["format"] in ("sell", "csr")
    t = res["table"]
    assert len(t) >= 12 and res["slice_iters_per_s"] > 0
    assert {e["order"] for e in t if e["format"] == "sell"} == {"rows", "tiles"}
    assert any(e["blocks_per_sm"] > 0 for e in t)
    assert max(e["slice_iters_per_s"] for e in t) == res["slice_iters_per_s"]
    c = inputs.make_case(128, 180, 6, seed=9, phantom="ellipsoids3d", noise="poisson", level=1e4)
    sino = torch.from_numpy(c.sino).cuda()
    auto = tomo.sirt(M, sino, 10, batch_width=0, fmt="auto")
    try:
        tomo.set_launch(order=res["order"], blocks_per_sm=res["blocks_per_sm"])
        expl = tomo.sirt(M, sino, 10, batch_width=res["batch_width"], fmt=res["format"])
        tomo.set_launch(order="rows", blocks_per_sm=3)
        other = tomo.sirt(M, sino, 10, batch_width=res["batch_width"], fmt=res["format"])
    finally:
        tomo.set_launch()
    assert torch.equal(auto, expl)   # same kernels, same sums: bit-identical
    assert torch.equal(auto, other)
    ref = oracle.sirt(A, AT, c.sino.reshape(6, -1), 10)
    assert per_slice_rel(auto.cpu().numpy(), ref).max() < 1e-4


def test_drop_csr_keeps_sell_paths():
    g, A, AT, M0 = pair(nx=64, nt=90)
    M = tomo.Matrix(64, 90, keep_csr=False)
    x = inputs.random_slices((3, 64, 64), seed=61)
    y = tomo.project(M, torch.from_numpy(x).cuda(), batch_width=4).cpu().numpy()
    assert per_slice_rel(y, A.apply(x)).max() < 1e-5
    with pytest.raises(_lib.TomoError):
        M.export_csr()
    with pytest.raises(_lib.TomoError):
        tomo.project(M, torch.from_numpy(x).cuda(), fmt="csr")
    assert M.autotune(3)["format"] == "sell"


def test_errors_are_reported():
    with pytest.raises(_lib.TomoError):
        tomo.Matrix(0, 10)
    g, A, AT, M = pair(nx=64, nt=45)
    with pytest.raises(_lib.TomoError):
        tomo.project(M, torch.zeros((3, 64, 64), device="cuda"), batch_width=3)
    with pytest.raises(_lib.TomoError):
        tomo.project(M, torch.zeros((1, 64, 64), device="cuda"), fmt="sell16")


TILE_GEOMS = [
    dict(nx=128, nt=180),                        # whole tiles, 180 angles (22.5 chunks of 8)
    dict(nx=37, nt=23, n_p=41, center=19.7),     # ragged tiles, shifted axis, 23 angles
    dict(nx=40, nt=7, ny=29, n_p=50),            # rectangular image, fewer angles than a chunk
    dict(nx=20, nt=9, ny=18, n_p=5),             # detector narrower than a tile's window
    GEOMS[3],                                    # given angles, two of them 1e-9 from 0 and pi
    GEOMS[4],                                    # one pixel, one ray
]


@pytest.mark.parametrize("values", ["bf16", "f16"])
@pytest.mark.parametrize("geom", TILE_GEOMS)
def test_tiled_at_same_bits(values, geom):
    """The 16-bit A^T in image tiles with each tile's detector window staged in
    shared memory (order "staged") adds every pixel's entries in the SELL
    pass's order: backprojection (19 slices: a full batch of 16 and a ragged
    one) and 10 SIRT iterations at width 16 give the bits of the row-order
    SELL pass; CGLS agrees within 1e-5 over 3 iterations (its FP64 norms are
    summed per block of another partition); backprojection equals the oracle
    applied to the same 16-bit values within 1e-5; a matrix built without the
    tiled copy runs order "staged" as the SELL pass."""
    g, A, AT, M = pair(values=values, **geom)
    assert M.has_at_tiles
    nx, ny, nt = geom["nx"], geom.get("ny", geom["nx"]), geom["nt"]
    _, AT16 = _oracle16(g, A, values)
    y = inputs.random_slices((19, nt, g.n_p), seed=71)
    yt = torch.from_numpy(y).cuda()
    x = inputs.random_slices((16, ny, nx), seed=72)
    sino = tomo.project(M, torch.from_numpy(x).cuda(), batch_width=16, fmt="sell16")
    out = {}
    try:
        for order in ("rows", "staged"):
            tomo.set_launch(order=order)
            out[order] = (tomo.backproject(M, yt, batch_width=16, fmt="sell16"),
                          tomo.sirt(M, sino, 10, batch_width=16, fmt="sell16"),
                          tomo.cgls(M, sino, 3, batch_width=16, fmt="sell16"))
        Mn = tomo.Matrix(nx, nt, n_p=geom.get("n_p"), n_y=geom.get("ny"), angles=geom.get("angles"),
                         center=geom.get("center"), values=values, at_tiles=False)
        assert not Mn.has_at_tiles
        tomo.set_launch(order="staged")
        xn = tomo.backproject(Mn, yt, batch_width=16, fmt="sell16")
    finally:
        tomo.set_launch()
    (br, sr, cr_), (bs, ss_, cs) = out["rows"], out["staged"]
    assert torch.equal(bs, br)
    assert torch.equal(ss_, sr)
    assert per_slice_rel(cs.cpu().numpy(), cr_.cpu().numpy()).max() < 1e-5
    assert torch.equal(xn, br)
    assert per_slice_rel(bs.cpu().numpy(), AT16.apply(y)).max() < 1e-5


def test_tiled_at_strip_model_and_auto_order():
    """The strip model (up to 3 bins per pixel and angle, wider windows) in
    the tiled form gives the row-order bits, and so does the default order
    (which takes the tiled form where it applies), one A^T launch per
    iteration."""
    M = tomo.Matrix(48, 30, n_p=56, values="bf16", model="strip")
    assert M.has_at_tiles
    x = inputs.random_slices((16, 48, 48), seed=73)
    sino = tomo.project(M, torch.from_numpy(x).cuda(), batch_width=16, fmt="sell16")
    try:
        tomo.set_launch(order="rows")
        ref = tomo.sirt(M, sino, 6, batch_width=16, fmt="sell16")
        tomo.set_launch(order="staged")
        st = tomo.sirt(M, sino, 6, batch_width=16, fmt="sell16")
    finally:
        tomo.set_launch()
    tm = tomo.new_timing()
    auto = tomo.sirt(M, sino, 6, batch_width=16, fmt="sell16", timing=tm)
    assert torch.equal(st, ref) and torch.equal(auto, ref)
    assert tm.launches[1] == 6


@pytest.mark.parametrize("values", ["bf16", "f16"])
@pytest.mark.parametrize("bands", [1, 3])
def test_pair_order_same_bits(values, bands):
    """The 16-bit A with its rows in pair order (each 8 rows: 2 angles x 4
    bins) gives the bits of the ray order: projection at widths 1, 4, 8 and 16
    (19 slices: full batches and a ragged one) and 10 SIRT iterations at width
    16, banded or not.  CGLS over 3 iterations, stand-alone and in the
    persistent batched solver, agrees within 1e-5 (its FP64 norms are summed
    per thread, and the threads hold other rays)."""
    kw = dict(n_p=72, n_y=40, values=values, col_blocks=bands)
    Mp, Mr = tomo.Matrix(48, 26, **kw), tomo.Matrix(48, 26, pair_order=False, **kw)
    x = torch.from_numpy(inputs.random_slices((19, 40, 48), seed=91)).cuda()
    for B in (1, 4, 8, 16):
        assert torch.equal(tomo.project(Mp, x, batch_width=B, fmt="sell16"),
                           tomo.project(Mr, x, batch_width=B, fmt="sell16")), B
    sino = tomo.project(Mr, x[:16].contiguous(), batch_width=16, fmt="sell16")
    assert torch.equal(tomo.sirt(Mp, sino, 10, batch_width=16, fmt="sell16"),
                       tomo.sirt(Mr, sino, 10, batch_width=16, fmt="sell16"))
    cp = tomo.cgls(Mp, sino, 3, batch_width=16, fmt="sell16").cpu().numpy()
    cr = tomo.cgls(Mr, sino, 3, batch_width=16, fmt="sell16").cpu().numpy()
    assert per_slice_rel(cp, cr).max() < 1e-5
    xp = tomo.cgls_batched([(Mp, sino[:5])], 3, batch_width=16, fmt="sell16")
    xr = tomo.cgls_batched([(Mr, sino[:5])], 3, batch_width=16, fmt="sell16")
    for a, b in zip(xp, xr):
        assert per_slice_rel(a.cpu().numpy(), b.cpu().numpy()).max() < 1e-5
    Mp.close()
    Mr.close()


def _oracle16(g, A, values):
    """The oracle's CSR pair with the 16-bit form's values (weights round(L a)
    times fl32(1/a), exact in FP64), so that the GPU's 16-bit kernels are held
    to their arithmetic alone."""
    import cgls_reference as cr
    v = cr.lowprec_values(A, g, values).astype(np.float64)
    A16 = oracle.CSR(A.rows, A.cols, A.row_ptr, A.col, v)
    return A16, A16.transpose()


@pytest.mark.parametrize("values", ["bf16", "f16"])
@pytest.mark.parametrize("geom,bands", [(dict(nx=96, nt=120), 3), (dict(nx=37, nt=23, n_p=41, center=19.7), 5),
                                        (dict(nx=40, nt=7, ny=29, n_p=50), 29)])
def test_banded_16bit_operator(values, geom, bands):
    """The 16-bit A stored as column bands (bands of image rows, one pass each,
    partial sums added in a workspace buffer): y = A x at widths 1, 4, 16
    (slice-major) and 8 (interleaved) equals the FP64 oracle applied to the same
    16-bit values within 1e-5, as does the unbanded form; x = A^T y too; CGLS
    over 3 iterations agrees with the unbanded form within 1e-4, in the
    stand-alone solver and in the persistent batched one."""
    g, A, AT, _ = pair(values=values, **geom)
    nx, ny, nt = geom["nx"], geom.get("ny", geom["nx"]), geom["nt"]
    kw = dict(n_p=geom.get("n_p"), n_y=geom.get("ny"), center=geom.get("center"), values=values)
    Mb = tomo.Matrix(nx, nt, col_blocks=bands, **kw)
    Mu = tomo.Matrix(nx, nt, **kw)
    A16, AT16 = _oracle16(g, A, values)
    x = inputs.random_slices((8, ny, nx), seed=61)
    y = inputs.random_slices((8, nt, g.n_p), seed=62)
    ref_y, ref_x = A16.apply(x), AT16.apply(y)
    xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    for M in (Mb, Mu):
        for B in (1, 4, 16):
            yd = tomo.project(M, xt, batch_width=B, fmt="sell16").cpu().numpy()
            assert per_slice_rel(yd, ref_y).max() < 1e-5, (B, M is Mb)
            xd = tomo.backproject(M, yt, batch_width=B, fmt="sell16").cpu().numpy()
            assert per_slice_rel(xd, ref_x).max() < 1e-5, (B, M is Mb)
        xi = xt.reshape(8, -1).t().contiguous()
        yi = tomo.project(M, xi, fmt="sell16", interleaved=True).t().cpu().numpy()
        assert per_slice_rel(yi, ref_y).max() < 1e-5
    sino = torch.from_numpy(np.ascontiguousarray(ref_y.astype(np.float32))).cuda()
    # the bands only change the order of FP32 sums, which CGLS amplifies (its
    # iterates part like two FP64 runs with different summation orders)
    cb = tomo.cgls(Mb, sino, 3, batch_width=4, fmt="sell16")
    cu = tomo.cgls(Mu, sino, 3, batch_width=4, fmt="sell16")
    assert per_slice_rel(cb.cpu().numpy(), cu.cpu().numpy()).max() < 1e-4
    # the persistent batched solver runs the banded A band by band (a grid
    # barrier between bands), mixed in one launch with an unbanded request
    xb = tomo.cgls_batched([(Mb, sino), (Mu, sino[:3])], 3, batch_width=4, fmt="sell16")
    assert per_slice_rel(xb[0].cpu().numpy(), cu.cpu().numpy()).max() < 1e-4
    assert per_slice_rel(xb[1].cpu().numpy(), cu[:3].cpu().numpy()).max() < 1e-4

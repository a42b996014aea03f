"""Parity at the full workload sizes, in the launch configurations the
benchmark uses, on outputs the FP64 oracle can compute (whole matrices where
the host holds them, sampled rows one by one otherwise) and on properties
that hold at any size.

  * 512x512 pixels, 360 angles, 64 slices (the benchmark workload): whole A
    and A^T bit-exact; 100 SIRT iterations on all 64 slices with the batch
    widths / formats the autotuner chooses between, two slices vs the oracle.
  * 2048x2048 pixels, 1024 angles, 16 slices, BF16 values: sampled rows of A
    and A^T bit-exact vs brute force, transpose consistency, sampled SpMM rows
    (FP32 CSR and BF16 SELL), 50 CGLS iterations with residual recompute.
  * 1024x1024 pixels, 720 angles, 32 slices: the autograd gradient of
    ||A x - b||^2 + 1e-3 TV(x) vs the matrix-free oracle gradient on 64
    random directions, and the adjoint identity.
"""
import numpy as np
import pytest

import oracle
from paper_2003_12677_b300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # the gpu marker is only run on a GPU machine
    pytest.skip("needs CUDA", allow_module_level=True)

import paper_2003_12677_b300 as tomo  # noqa: E402


_cases = {}


def case_of(name):
    if name not in _cases:
        _cases[name] = inputs.workload_case(name)
    return _cases[name]


def rel(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


# ---------------------------------------------------------------------------
# 512 x 512 x 360, 64 slices
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def bench_pair():
    g = oracle.Geometry(512, 512, 512, 360)
    A = oracle.build_matrix(g)
    M = tomo.Matrix(512, 360)
    yield g, A, M
    M.close()


def test_bench_matrix_bitexact(bench_pair):
    g, A, M = bench_pair
    assert M.nnz == A.nnz
    rp, col, val = M.export_csr()
    np.testing.assert_array_equal(rp, A.row_ptr)
    np.testing.assert_array_equal(col, A.col)
    np.testing.assert_array_equal(val, A.val.astype(np.float32))
    del rp, col, val
    AT = A.transpose()
    rp, col, val = M.export_csr(transpose=True)
    np.testing.assert_array_equal(rp, AT.row_ptr)
    np.testing.assert_array_equal(col, AT.col)
    np.testing.assert_array_equal(val, AT.val.astype(np.float32))


@pytest.mark.parametrize("B,fmt", [(64, "csr"), (16, "sell")])
def test_bench_sirt_sampled_slices(bench_pair, B, fmt):
    g, A, M = bench_pair
    case = case_of("sirt_512x360_b64")
    x = tomo.sirt(M, torch.from_numpy(case.sino).cuda(), 100, batch_width=B, fmt=fmt).cpu().numpy()
    AT = A.transpose()
    pick = [0, 37]
    ref = oracle.sirt(A, AT, case.sino[pick].reshape(2, -1), 100)
    for k, s in enumerate(pick):
        assert rel(x[s], ref[k]) < 1e-4


# ---------------------------------------------------------------------------
# 2048 x 2048 x 1024, 16 slices, BF16 values
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def big():
    g = oracle.Geometry(2048, 2048, 2048, 1024)
    M = tomo.Matrix(2048, 1024, values="bf16", fp32_sell=False)
    yield g, M
    M.close()
    torch.cuda.empty_cache()


RAYS = [0, 2047, 1024, 300 * 2048 + 5, 256 * 2048 + 1000, 511 * 2048 + 2040, 768 * 2048 + 17,
        1023 * 2048 + 1023, 700 * 2048 + 1500]


def test_big_rows_bitexact_and_transpose_consistent(big):
    g, M = big
    assert M.nnz > 5.0e9
    for i in RAYS:
        rp, col, val = M.export_rows(i, i + 1)
        c2, v2 = oracle.row(g, i)
        np.testing.assert_array_equal(col, c2)
        np.testing.assert_array_equal(val, v2.astype(np.float32))
        for j, v in list(zip(col, val))[:: max(1, len(col) // 12)]:
            trp, tcol, tval = M.export_rows(int(j), int(j) + 1, transpose=True)
            k = np.searchsorted(tcol, i)
            assert tcol[k] == i and tval[k] == v
    for j in [0, 2047, 2048 * 1024 + 1024, 2048 * 2048 - 1, 777 * 2048 + 3]:
        trp, tcol, tval = M.export_rows(j, j + 1, transpose=True)
        c2, v2 = oracle.pixel_row(g, j)
        np.testing.assert_array_equal(tcol, c2)
        np.testing.assert_array_equal(tval, v2.astype(np.float32))


@pytest.mark.parametrize("fmt,tol", [("csr", 1e-5), ("sell16", 5e-3)])
def test_big_spmm_sampled_rows(big, fmt, tol):
    g, M = big
    case = case_of("cgls_2048x1024_b16")
    x = torch.from_numpy(case.phantom).cuda()
    y = tomo.project(M, x, batch_width=16, fmt=fmt).cpu().numpy().reshape(16, -1)
    xf = case.phantom.reshape(16, -1).astype(np.float64)
    got, ref = [], []
    for i in RAYS:
        c2, v2 = oracle.row(g, i)
        ref.append(xf[:, c2] @ v2)
        got.append(y[:, i])
    assert rel(got, ref) < tol
    # A^T rows
    r = inputs.random_slices((16, 1024, 2048), seed=5)
    xb = tomo.backproject(M, torch.from_numpy(r).cuda(), batch_width=16, fmt=fmt).cpu().numpy().reshape(16, -1)
    rf = r.reshape(16, -1).astype(np.float64)
    got, ref = [], []
    for j in [0, 2048 * 1024 + 1024, 2048 * 2048 - 1, 777 * 2048 + 3, 1500 * 2048 + 900]:
        c2, v2 = oracle.pixel_row(g, j)
        ref.append(rf[:, c2] @ v2)
        got.append(xb[:, j])
    assert rel(got, ref) < tol


def test_big_cgls_bf16_50_iterations(big):
    """The 16-slice BF16 workload: 50 CGLS iterations with the residual
    recomputed every 10; the residual norm stays finite and never increases
    beyond FP32 noise."""
    g, M = big
    case = case_of("cgls_2048x1024_b16")
    x, h = tomo.cgls(M, torch.from_numpy(case.sino).cuda(), 50, recompute_every=10, history=True,
                     batch_width=16, fmt="sell16")
    h = h.cpu().numpy()
    assert np.all(np.isfinite(h)) and torch.isfinite(x).all()
    assert np.all(h[1:] <= h[:-1] * (1 + 1e-3))
    assert np.all(h[-1] < 0.5 * h[0])


def test_big_cgls_bf16_against_the_oracle(big):
    """The same workload and launch configuration (16 slices, width 16, BF16
    values, residual recomputed every 10) against the FP64 oracle, on what the
    oracle can compute at this size (the matrix-free oracle takes ~20 s per
    iteration on the host):

      * the first three iterates of slice 0 at the 1,024 seeded pixels the
        stored oracle run kept (tests/golden/cgls_2048x1024_slice0.json) within
        2e-4 (the BF16 values alone move them by ~5e-5: round-off 2^-9 on the
        ramp entries, averaged over ~2,400 entries a row);
      * one step from the GPU's own state after 10 and after 40 iterations
        against one matrix-free FP64 oracle step from that state (slice 0): x
        within 1e-4, r and p within 1e-3, gamma within 1e-3 (the BF16 operator
        against the exact one, the same bound);
      * the data fit ||b - A x_k|| of slice 0 reaches the oracle's 50-iteration
        value (stored, to 1e-4) within 60 iterations (reading of the CGLS
        precision: FP32 arithmetic lags the FP64 trajectory by a few iterations)."""
    import json
    import os
    g, M = big
    case = case_of("cgls_2048x1024_b16")
    sino = torch.from_numpy(case.sino).cuda()
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "cgls_2048x1024_slice0.json")) as f:
        gold = json.load(f)
    target = gold["resnorm"][49] * (1 + 1e-4)
    idx = torch.tensor(gold["sample_index"], device="cuda")
    b0 = sino[:1].contiguous()
    kw = dict(batch_width=16, fmt="sell16")
    x, st = tomo.cgls(M, sino, 0, return_state=True, **kw)
    reached = None
    for k in range(1, 61):
        x, st = tomo.cgls(M, sino, 1, recompute_every=1 if k % 10 == 0 else 0, resume=st, return_state=True, **kw)
        if k <= 3:
            ref = np.array([float(v) for v in gold["samples"][str(k)]])
            got = x[0].reshape(-1)[idx].double().cpu().numpy()
            assert rel(got, ref) < 2e-4, k
        if k in (10, 40):
            _, st1 = tomo.cgls(M, sino, 1, resume=st, return_state=True, **kw)
            s0 = {n: st[n][:1].double().cpu().numpy().reshape(1, -1) for n in ("x", "r", "p")}
            xo, ro, po, go, _fo, _h = oracle.cgls_resume_mf(g, s0["x"], s0["r"], s0["p"], st["gamma"][:1].cpu().numpy(),
                                                        st["frozen"][:1].cpu().numpy(), 1)
            assert rel(st1["x"][0].cpu().numpy(), xo) < 1e-4, k
            assert rel(st1["r"][0].cpu().numpy(), ro) < 1e-3, k
            assert rel(st1["p"][0].cpu().numpy(), po) < 1e-3, k
            assert abs(float(st1["gamma"][0]) - float(go[0])) <= 1e-3 * float(go[0]), k
        fit = float(tomo.residual_norm(M, b0, x[:1].contiguous())[0])
        if k >= 50 and fit <= target:
            reached = k
            break
    assert reached is not None and reached <= 60, (reached, fit, target)


# ---------------------------------------------------------------------------
# 1024 x 1024 x 720, 32 slices: gradient through autograd
# ---------------------------------------------------------------------------

def test_gradient_1024_vs_matrix_free_oracle():
    n, nt, nz = 1024, 720, 32
    g = oracle.Geometry(n, n, n, nt)
    M = tomo.Matrix(n, nt)
    case = case_of("gd_1024x720_b32")
    rng = np.random.default_rng(44)
    x0 = (case.phantom + 0.1 * rng.standard_normal(case.phantom.shape)).astype(np.float32)
    xt = torch.from_numpy(x0).cuda().requires_grad_(True)
    b = torch.from_numpy(case.sino).cuda()
    r = tomo.radon(xt, M) - b
    loss = (r * r).sum() + 1e-3 * tomo.tv_loss(xt, 1e-3)
    loss.backward()
    gd = xt.grad.double().cpu().numpy().reshape(nz, -1)
    f, gref = oracle.loss_grad_mf(g, x0.reshape(nz, -1), case.sino.reshape(nz, -1), 1e-3, 1e-3)
    assert abs(loss.item() - f) <= 1e-4 * abs(f)
    gn = np.linalg.norm(gref)
    for _ in range(64):
        v = rng.standard_normal(gd.shape)
        v /= np.linalg.norm(v)
        assert abs(float(np.sum(gd * v)) - float(np.sum(gref * v))) <= 1e-4 * gn
    # adjoint identity at full size
    xr = torch.from_numpy(inputs.random_slices((nz, n, n), 1)).cuda()
    yr = torch.from_numpy(inputs.random_slices((nz, nt, n), 2)).cuda()
    lhs = torch.sum(tomo.project(M, xr).double() * yr.double()).item()
    rhs = torch.sum(xr.double() * tomo.backproject(M, yr).double()).item()
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)
    M.close()

"""BB-step SIRT with Hamming preconditioning (Sec. 3.1) on the GPU vs the FP64
oracle, through the C ABI.

Bars: the first step (the FBP, Sec. 2.1) within 1e-5 relative L2 per slice
(FP32 SpMM and filter); whole trajectories within 1e-4 over 10 iterations (an
FP32 emulation of the recurrence stays within 1e-6 there and drifts past 1e-4
only after ~17 iterations, as BB steps amplify rounding); every step of 40 as
one oracle step from the GPU's own state (x within 1e-5; the gradient within a
bound that follows the cancellation in b - A x)."""
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


def pair(nx, nt, n_p=None, ny=None, center=None, values="f32"):
    key = (nx, nt, n_p, ny, center, values)
    if key not in _cache:
        g = oracle.Geometry(nx, nx if ny is None else ny, nx if n_p is None else n_p, nt, None, center)
        A = oracle.build_matrix(g)
        M = tomo.Matrix(nx, nt, n_p=n_p, n_y=ny, center=center, values=values)
        _cache[key] = (g, A, A.transpose(), M)
    return _cache[key]


def case_128(nz):
    c = inputs.make_case(128, 180, nz, seed=501, phantom="ellipsoids3d", noise="poisson", level=1e5)
    return c.sino


GEOS = [dict(nx=128, nt=180), dict(nx=96, nt=120, n_p=101, ny=80, center=49.3), dict(nx=33, nt=17)]


@pytest.mark.parametrize("geo", GEOS)
@pytest.mark.parametrize("B", [1, 4, 16])
def test_first_step_is_the_oracle_fbp(geo, B):
    g, A, AT, M = pair(**geo)
    nz = 5
    b = inputs.random_slices((nz, g.n_theta, g.n_p), seed=7)
    x = tomo.sirt_bb(M, torch.from_numpy(b).cuda(), 1, batch_width=B)
    ref, h = oracle.sirt_bb(A, AT, g.n_p, b.reshape(nz, -1), 1)
    assert per_slice_rel(x.cpu().numpy(), ref).max() < 1e-5


@pytest.mark.parametrize("B,fmt", [(1, "csr"), (4, "sell"), (16, "sell"), (64, "csr")])
def test_trajectory_10_iterations(B, fmt):
    g, A, AT, M = pair(nx=128, nt=180)
    sino = case_128(6)
    x, h = tomo.sirt_bb(M, torch.from_numpy(sino).cuda(), 10, history=True, batch_width=B, fmt=fmt)
    ref, href = oracle.sirt_bb(A, AT, 128, sino.reshape(6, -1), 10)
    assert per_slice_rel(x.cpu().numpy(), ref).max() < 1e-4
    np.testing.assert_allclose(h.cpu().numpy(), href, rtol=1e-4)


EPS32 = 2.0 ** -24


@pytest.mark.parametrize("B", [4, 32])
def test_every_step_matches_an_oracle_step(B):
    """40 single-iteration calls, each resumed from the state the previous one
    returned: each equals one FP64 oracle step from that state.

    The bound follows the arithmetic.  The step recomputes r = b - A x in FP32
    from terms of size ||b||, so r carries a white error of about
    eps32 ||b||; g = A^T P^T P r passes that error through the ramp filter,
    which lifts white noise more than the residual itself.  With gain(v) =
    ||A^T P^T P v|| / ||v|| (oracle operators), g's relative error is about
    eps32 (||b|| / ||r||) gain(white) / gain(r) times a small constant; alpha
    follows g, and x inherits the error of alpha g in proportion to the step
    ||x_new - x|| / ||x_new||."""
    g, A, AT, M = pair(nx=128, nt=180)
    sino = case_128(3)
    b64 = sino.reshape(3, -1).astype(np.float64)
    st_b = torch.from_numpy(sino).cuda()
    rng = np.random.default_rng(5)
    D = oracle.ramp_response(128)
    gain = lambda v: np.linalg.norm(oracle.backproject(AT, oracle.ramp_filter(v, 128, D)), axis=1) / \
        np.linalg.norm(v, axis=1)  # noqa: E731
    gain_white = gain(rng.standard_normal((3, A.rows)))
    x, st = tomo.sirt_bb(M, st_b, 0, batch_width=B, return_state=True)
    worst = 0.0
    for k in range(40):
        x1, st1 = tomo.sirt_bb(M, st_b, 1, batch_width=B, resume=st, return_state=True)
        x_prev = st["x"].double().cpu().numpy().reshape(3, -1)
        ref = oracle.sirt_bb_resume(A, AT, 128, b64, x_prev,
                                    None if k == 0 else st["g"].double().cpu().numpy(),
                                    None if k == 0 else st["alpha"].cpu().numpy(),
                                    None if k == 0 else st["frozen"].cpu().numpy(), 1)
        r = b64 - oracle.project(A, x_prev)
        amp = np.linalg.norm(b64, axis=1) / np.linalg.norm(r, axis=1) * gain_white / gain(r)
        tol = 1e-6 + 16 * EPS32 * amp
        err_g = per_slice_rel(st1["g"].cpu().numpy(), ref[1])
        worst = max(worst, float(np.max(err_g / (EPS32 * amp))))
        assert np.all(err_g < tol), (k, err_g, tol, worst)
        assert np.all(np.abs(st1["alpha"].cpu().numpy() - ref[2]) <= 2 * tol * np.abs(ref[2])), k
        step = np.linalg.norm(ref[0] - x_prev, axis=1) / np.linalg.norm(ref[0], axis=1)
        assert np.all(per_slice_rel(x1.cpu().numpy(), ref[0]) < 1e-6 + 4 * tol * step), k
        np.testing.assert_array_equal(st1["frozen"].cpu().numpy() != 0, ref[3])
        st = st1
    print("largest g error in units of eps32 * amplification:", worst)


def test_resume_and_graph_are_bitwise():
    g, A, AT, M = pair(nx=128, nt=180)
    b = torch.from_numpy(case_128(5)).cuda()
    x9 = tomo.sirt_bb(M, b, 9, batch_width=4)
    x9n = tomo.sirt_bb(M, b, 9, batch_width=4, use_graph=False)
    assert torch.equal(x9, x9n)
    x4, st = tomo.sirt_bb(M, b, 4, batch_width=4, return_state=True)
    x5 = tomo.sirt_bb(M, b, 5, batch_width=4, resume=st)
    assert torch.equal(x5, x9)


def test_zero_data_freezes_and_x0_is_used():
    g, A, AT, M = pair(nx=33, nt=17)
    z = torch.zeros((2, 17, 33), device="cuda")
    x, h = tomo.sirt_bb(M, z, 4, history=True, batch_width=2)
    assert torch.all(x == 0) and torch.all(h == 0)
    x0 = torch.rand((2, 33, 33), device="cuda")
    b = torch.from_numpy(inputs.random_slices((2, 17, 33), 3)).cuda()
    x = tomo.sirt_bb(M, b, 3, x0=x0, batch_width=2)
    ref = oracle.sirt_bb_resume(A, AT, 33, b.double().cpu().numpy().reshape(2, -1),
                                x0.double().cpu().numpy().reshape(2, -1), None, None, None, 3)[0]
    assert per_slice_rel(x.cpu().numpy(), ref).max() < 1e-4


@pytest.mark.parametrize("values", ["bf16", "f16"])
def test_16bit_values(values):
    """BB-SIRT on 16-bit values: 5 iterations within 1e-4 of the FP64 oracle
    run on the same 16-bit values (weights round(L a) times fl32(1/a))."""
    import cgls_reference as cr
    g, A, AT, M = pair(nx=128, nt=180, values=values)
    v = cr.lowprec_values(A, g, values).astype(np.float64)
    A16 = oracle.CSR(A.rows, A.cols, A.row_ptr, A.col, v)
    sino = case_128(4)
    x = tomo.sirt_bb(M, torch.from_numpy(sino).cuda(), 5, batch_width=4, fmt="sell16")
    ref, _ = oracle.sirt_bb(A16, A16.transpose(), 128, sino.reshape(4, -1), 5)
    assert per_slice_rel(x.cpu().numpy(), ref).max() < 1e-4


def test_converges_faster_than_classical_sirt():
    """The paper's claim for this SIRT (Sec. 3.1): about 10x faster
    convergence.  Here: 5 BB-preconditioned iterations reach a lower data
    residual than 100 classical SIRT iterations on the 128x128, 180-angle case
    (BB is not monotone: at 10 iterations one slice sits on a spike)."""
    g, A, AT, M = pair(nx=128, nt=180)
    b = torch.from_numpy(case_128(4)).cuda()
    xb = tomo.sirt_bb(M, b, 5, batch_width=4)
    xs = tomo.sirt(M, b, 100, batch_width=4)
    rb = torch.linalg.vector_norm((tomo.project(M, xb) - b).reshape(4, -1), dim=1)
    rs = torch.linalg.vector_norm((tomo.project(M, xs) - b).reshape(4, -1), dim=1)
    assert torch.all(rb < rs)

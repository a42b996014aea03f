"""CGLS across value precisions on the GPU, against the FP64 oracle (Sec. 2.1).

CGLS trajectories are not reproducible iterate by iterate past the first few
in any precision on these systems (tests/test_cgls_precision.py pins this on
the CPU: two FP64 runs with different summation orders part by more than
1e-3).  So the forms are held to the oracle three ways:

  * the first four iterates: FP32 forms within 1e-4 of the FP64 oracle; 16-bit
    forms within 1e-4 of the FP64 oracle run on the same 16-bit values;
  * every later step one at a time (test_gpu_parity.py);
  * the data fit ||b - A x_k||, the quantity CGLS minimises: every form must
    reach the oracle's 50-iteration data fit (to 1e-4) within 65 iterations,
    and the 16-bit forms within 3 iterations of the plain FP32 CSR SpMV form:
    reduced precision costs no accuracy at equal data fit.

The data fit of a GPU iterate comes from tomo_residual_norm (FP64
accumulation), itself checked against the oracle here.  The per-iterate table
(relative L2 to the oracle's iterate, data fit over the oracle's) is printed
(pytest -s)."""
import numpy as np
import pytest

import oracle
from paper_2003_12677_b300 import inputs

import cgls_reference as cr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs CUDA", allow_module_level=True)

import paper_2003_12677_b300 as tomo  # noqa: E402

WALK = 70
TARGET = 50
REPORT = (1, 2, 3, 4, 5, 10, 20, 30, 40, 50, 60)

# (label, value dtype of the build, fmt, batch width, recompute every, recompute with FP32 values)
FORMS = [("plain FP32 CSR SpMV", "f32", "csr", 1, 0, False),
         ("FP32 SELL-32", "f32", "sell", 2, 0, False),
         ("BF16 SELL-16", "bf16", "sell16", 2, 0, False),
         ("F16 SELL-16", "f16", "sell16", 2, 0, False),
         ("BF16 SELL-16, recompute/10 FP32 values", "bf16", "sell16", 2, 10, True)]


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def _case(n, nt):
    if n == 128:
        c = inputs.make_case(128, 180, 2, seed=12677 + 1, phantom="ellipses2d", noise="poisson", level=1e5)
    else:
        c = inputs.workload_case("sirt_512x360_b64", slices=[0])
    return c.sino.reshape(c.n_z, -1)


def _oracle_walk(A, AT, b, iters):
    """The oracle's iterates x_1 .. x_iters of every slice, (iters, nz, cols)."""
    nz = b.shape[0]
    x = np.zeros((nz, A.cols))
    r = np.array(b, np.float64)
    s = AT.apply(r)
    p = s.copy()
    gamma = np.array([sum(v * v for v in s[z]) for z in range(nz)])
    frozen = np.zeros(nz, np.int32)
    out = []
    for _ in range(iters):
        x, r, p, gamma, frozen, _h = oracle.cgls_resume(A, AT, x, r, p, gamma, frozen, 1)
        out.append(x.copy())
    return np.stack(out)


def _gpu_walk(M, sino, fmt, B, recompute, fp32):
    """Data fits ||b - A x_k|| (k = 1 .. WALK, per slice) and the first iterates."""
    x, st = tomo.cgls(M, sino, 0, batch_width=B, fmt=fmt, return_state=True)
    fits, first = [], []
    for k in range(1, WALK + 1):
        rc = 1 if (recompute and k % recompute == 0) else 0   # the recompute of a straight run at k
        x, st = tomo.cgls(M, sino, 1, recompute_every=rc, batch_width=B, fmt=fmt, resume=st, return_state=True,
                          recompute_fp32=fp32)
        fits.append(tomo.residual_norm(M, sino, x).cpu().numpy())
        if k <= 4 or k in REPORT:
            first.append((k, x.cpu().numpy().reshape(x.shape[0], -1)))
    return np.array(fits), dict(first)


@pytest.mark.parametrize("n,nt", [(128, 180), (512, 360)])
def test_cgls_precisions_against_the_oracle(n, nt):
    g = oracle.Geometry(n, n, n, nt)
    A = oracle.build_matrix(g)
    AT = A.transpose()
    b = _case(n, nt)
    nz = b.shape[0]
    ref = _oracle_walk(A, AT, b, WALK)                    # (WALK, nz, cols)
    S64, _ = cr.csr_pair(A)
    ref_fit = np.array([[np.linalg.norm(b[z] - S64 @ ref[k, z]) for z in range(nz)] for k in range(WALK)])
    target = ref_fit[TARGET - 1] * (1 + 1e-4)
    sino = torch.from_numpy(np.ascontiguousarray(b.reshape(nz, nt, n))).cuda()
    mats = {}
    lp_ref = {}
    table, reach = [], {}
    for label, values, fmt, B, rc, fp32 in FORMS:
        if values not in mats:
            mats[values] = tomo.Matrix(n, nt, values=values)
        M = mats[values]
        fits, xs = _gpu_walk(M, sino, fmt, B, rc, fp32)
        # the data-fit kernel against FP64 products of the same iterates
        for k in (1, TARGET):
            xk = xs[k]
            exact = np.array([np.linalg.norm(b[z] - S64 @ xk[z]) for z in range(nz)])
            np.testing.assert_allclose(fits[k - 1], exact, rtol=1e-5, err_msg=label)
        # the first iterates
        if fmt == "sell16":
            if values not in lp_ref:
                v = cr.lowprec_values(A, g, values).astype(np.float64)
                A16 = oracle.CSR(A.rows, A.cols, A.row_ptr, A.col, v)
                lp_ref[values] = _oracle_walk(A16, A16.transpose(), b, 4)
            base = lp_ref[values]
        else:
            base = ref[:4]
        for k in range(1, 5):
            if rc and k % rc == 0:
                continue
            for z in range(nz):
                assert _rel(xs[k][z], base[k - 1, z]) < 1e-4, (label, k, z)
        ks = [cr.iters_to_fit(fits[:, z], target[z]) for z in range(nz)]
        reach[label] = ks
        rows = []
        for k in REPORT:
            if k in xs:
                rows.append((k, max(_rel(xs[k][z], ref[k - 1, z]) for z in range(nz)),
                             float(np.max(fits[k - 1] / ref_fit[k - 1]))))
        table.append((label, ks, rows))
    print("\nCGLS %dx%d, %d angles, %d slice(s): oracle 50-iteration data fit %s" % (n, n, nt, nz, ref_fit[TARGET - 1]))
    for label, ks, rows in table:
        print("  %-40s iterations to reach it: %s" % (label, ks))
        print("    " + "  ".join("k=%d: relL2 %.1e fit/oracle %.5f" % r for r in rows))
    plain = reach["plain FP32 CSR SpMV"]
    for label, ks in reach.items():
        if "recompute" in label:
            continue          # reported only: the FP32-value recompute is a reading under test, not a bar
        assert all(k is not None and k <= 65 for k in ks), (label, ks)
        if "16" in label:
            assert all(abs(a - p) <= 3 for a, p in zip(ks, plain)), (label, ks, plain)


def test_residual_norm_is_the_fp64_data_fit_of_the_fp32_operator():
    """tomo_residual_norm equals the FP64 data fit of the FP32-rounded operator
    to 1e-12 (exact products, FP64 sums in another order), for 3 slices."""
    g = oracle.Geometry(96, 96, 101, 75, center=49.3)
    A = oracle.build_matrix(g)
    A32 = oracle.CSR(A.rows, A.cols, A.row_ptr, A.col, A.val.astype(np.float32).astype(np.float64))
    rng = np.random.default_rng(5)
    x = rng.random((3, A.cols)).astype(np.float32)
    b = (A32.apply(x) + rng.standard_normal((3, A.rows))).astype(np.float32)
    M = tomo.Matrix(96, 75, n_p=101, center=49.3)
    got = tomo.residual_norm(M, torch.from_numpy(b).cuda(), torch.from_numpy(x).cuda()).cpu().numpy()
    exact = np.linalg.norm(b - A32.apply(x), axis=1)
    np.testing.assert_allclose(got, exact, rtol=1e-12)


def _batched_walk(pairs, fmt, fit_mats, iters):
    """Data fits ||b - A x_k|| (k = 1 .. iters) of every request's slices, and
    its first iterate: the persistent batched solver, one launch per
    iteration, resumed from the previous state."""
    xs, states = tomo.cgls_batched(pairs, 0, batch_width=4, fmt=fmt, return_state=True)
    fits, first = [], None
    for k in range(1, iters + 1):
        xs, states = tomo.cgls_batched(pairs, 1, batch_width=4, fmt=fmt, resume=states, return_state=True)
        fits.append([tomo.residual_norm(fit_mats[i], s, x).cpu().numpy() for i, ((_, s), x) in enumerate(zip(pairs, xs))])
        if k == 1:
            first = [x.cpu().numpy().reshape(x.shape[0], -1) for x in xs]
    return fits, first


def test_batched_precisions_at_equal_data_fit():
    """The uneven batch (one persistent launch per iteration for requests of
    three geometries and 1-3 slices) with FP32 and with BF16 values: every
    slice reaches the FP64 oracle's 30-iteration data fit (to 1e-4) within 40
    iterations in both precisions, BF16 within 3 iterations of FP32; the FP32
    form's first iterate is within 1e-4 of the oracle's."""
    geos = [(64, 90, 1, 31), (96, 60, 3, 32), (128, 180, 2, 33)]
    reqs32, reqs16, fit_mats, refs = [], [], [], []
    for n, nt, nz, seed in geos:
        g = oracle.Geometry(n, n, n, nt)
        A = oracle.build_matrix(g)
        AT = A.transpose()
        c = inputs.make_case(n, nt, nz, seed=seed, phantom="ellipsoids3d", noise="poisson", level=1e5)
        b = c.sino.reshape(nz, -1)
        walk = _oracle_walk(A, AT, b, 30)
        S64, _ = cr.csr_pair(A)
        refs.append((np.array([np.linalg.norm(b[z] - S64 @ walk[29, z]) for z in range(nz)]), walk[0]))
        sino = torch.from_numpy(np.ascontiguousarray(c.sino)).cuda()
        M32, M16 = tomo.Matrix(n, nt), tomo.Matrix(n, nt, values="bf16")
        reqs32.append((M32, sino))
        reqs16.append((M16, sino))
        fit_mats.append(M32)
    f32, first32 = _batched_walk(reqs32, "sell", fit_mats, 40)
    f16, _ = _batched_walk(reqs16, "sell16", fit_mats, 40)
    for i, (target, x1) in enumerate(refs):
        for z in range(len(target)):
            k32 = cr.iters_to_fit(np.array([f[i][z] for f in f32]), target[z] * (1 + 1e-4))
            k16 = cr.iters_to_fit(np.array([f[i][z] for f in f16]), target[z] * (1 + 1e-4))
            print("  request %d slice %d (%dx%d, %d angles): FP32 %s, BF16 %s iterations" %
                  (i, z, geos[i][0], geos[i][0], geos[i][1], k32, k16))
            assert k32 is not None and k16 is not None and k32 <= 40 and k16 <= 40
            assert abs(k16 - k32) <= 3
            assert _rel(first32[i][z], x1[z]) < 1e-4

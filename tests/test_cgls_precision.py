"""The precision reading of CGLS (Sec. 2.1), pinned on the CPU.

CGLS iterates beyond the first few are not a reproducible function of the
data in any floating-point precision on these systems: the recurrence loses
orthogonality, and where the FP64 run and a perturbed run then place their
"ghost" directions differs.  So whole trajectories are compared only over the
first iterations, every later step is compared one step at a time (the GPU
tests), and accuracy across precisions is measured by the quantity CGLS
minimises: the data fit ||b - A x||.  These pins establish, with the FP64
oracle and independent numpy recurrences only:

  1. two FP64 runs with different summation orders agree to 1e-11 over the
     first five iterations and then differ by more than 1e-3;
  2. an FP32 run (FP32 vectors and products, FP64 dots: the GPU arithmetic)
     tracks the oracle to 1e-5 over the first four iterations, then drifts by
     more than 1e-3, and still reaches the oracle's 50-iteration data fit
     (to 1e-4) within 60 iterations;
  3. 16-bit matrix values (bf16 and f16 with the per-angle scale) reach that
     data fit in as many iterations as FP32 values, within two;
  4. recomputing the residual with the FP32 values while the recurrence runs
     on the 16-bit ones does not reach it sooner: the mismatch between the
     two operators enters r and spoils the conjugacy, so the recompute keeps
     the operator of the recurrence.
"""
import numpy as np
import pytest

import oracle
from paper_2003_12677_b300 import inputs

import cgls_reference as cr

TARGET_ITERS = 50


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


_cache = {}


def _system(n, nt):
    if (n, nt) not in _cache:
        g = oracle.Geometry(n, n, n, nt)
        A = oracle.build_matrix(g)
        AT = A.transpose()
        c = inputs.make_case(n, nt, 1, seed=12677 + 1, phantom="ellipses2d", noise="poisson", level=1e5)
        b = c.sino.reshape(-1).astype(np.float64)
        # the oracle's iterates x_1 .. x_60, one resumed step at a time
        x = np.zeros((1, A.cols))
        r = b[None].copy()
        s = AT.apply(r)
        p = s.copy()
        gamma = np.array([sum(v * v for v in s[0])])
        frozen = np.zeros(1, np.int32)
        ref = []
        for _ in range(60):
            x, r, p, gamma, frozen, _h = oracle.cgls_resume(A, AT, x, r, p, gamma, frozen, 1)
            ref.append(x[0].copy())
        _cache[(n, nt)] = (g, A, b, ref)
    return _cache[(n, nt)]


@pytest.mark.parametrize("n,nt", [(64, 90), (128, 180)])
def test_fp64_trajectories_part_after_the_first_iterations(n, nt):
    g, A, b, ref = _system(n, nt)
    S, ST = cr.csr_pair(A)
    xs = cr.textbook_cgls(S, ST, b, TARGET_ITERS, np.float64)
    d = [_rel(xs[k], ref[k]) for k in range(TARGET_ITERS)]
    assert max(d[:5]) < 1e-11, d[:5]
    assert max(d) > 1e-3, max(d)


def test_fp32_drifts_but_reaches_the_fp64_data_fit():
    g, A, b, ref = _system(64, 90)
    S32, ST32 = cr.csr_pair(A, A.val.astype(np.float32), np.float32)
    S64, _ = cr.csr_pair(A)
    xs = cr.textbook_cgls(S32, ST32, b, 60, np.float32)
    d = [_rel(xs[k], ref[k]) for k in range(TARGET_ITERS)]
    assert max(d[:4]) < 1e-5, d[:4]
    assert max(d) > 1e-3, max(d)
    target = np.linalg.norm(b - S64 @ ref[TARGET_ITERS - 1]) * (1 + 1e-4)
    k = cr.iters_to_fit(cr.data_fit(S64, b, xs), target)
    assert k is not None and TARGET_ITERS <= k <= 60, k


def test_16bit_values_reach_the_data_fit_as_fast_as_fp32():
    g, A, b, ref = _system(64, 90)
    S64, _ = cr.csr_pair(A)
    target = np.linalg.norm(b - S64 @ ref[TARGET_ITERS - 1]) * (1 + 1e-4)
    S32, ST32 = cr.csr_pair(A, A.val.astype(np.float32), np.float32)
    k32 = cr.iters_to_fit(cr.data_fit(S64, b, cr.textbook_cgls(S32, ST32, b, 70, np.float32)), target)
    for kind in ("bf16", "f16"):
        v = cr.lowprec_values(A, g, kind)
        assert 0 < _rel(v.astype(np.float64), A.val) < (2e-3 if kind == "bf16" else 3e-4)
        S16, ST16 = cr.csr_pair(A, v, np.float32)
        k16 = cr.iters_to_fit(cr.data_fit(S64, b, cr.textbook_cgls(S16, ST16, b, 70, np.float32)), target)
        assert k16 is not None and abs(k16 - k32) <= 2, (kind, k16, k32)


def test_fp32_value_recompute_does_not_win_back_the_data_fit():
    g, A, b, ref = _system(64, 90)
    S64, _ = cr.csr_pair(A)
    target = np.linalg.norm(b - S64 @ ref[TARGET_ITERS - 1]) * (1 + 1e-4)
    S32, _ = cr.csr_pair(A, A.val.astype(np.float32), np.float32)
    S16, ST16 = cr.csr_pair(A, cr.lowprec_values(A, g, "bf16"), np.float32)
    same = cr.iters_to_fit(cr.data_fit(S64, b, cr.textbook_cgls(S16, ST16, b, 90, np.float32, 10)), target)
    fp32 = cr.iters_to_fit(cr.data_fit(S64, b, cr.textbook_cgls(S16, ST16, b, 90, np.float32, 10, S32)), target)
    assert same is not None and fp32 is not None
    assert fp32 >= same, (fp32, same)

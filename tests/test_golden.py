"""Golden fixtures (tests/golden/*.json, written by tests/golden/make_golden.py
from the FP64 oracle only).

CPU: the oracle still reproduces every stored value bit for bit (structure,
chord lengths) or to FP64 rounding (SIRT / CGLS iterates), and the fixtures
carry the facts a reader can check by hand (theta = 0 rows of the square grid:
one unit chord per pixel of a column).  GPU: the library builds the same
structure bit for bit, FP32-rounded values, and SIRT / CGLS iterates within
the FP32 tolerances of Sec. 2.1's solvers against the stored FP64 ones."""
import glob
import json
import os

import numpy as np
import pytest

import oracle

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
# the small fixtures of make_golden.py (cgls_*_slice0.json are data-fit histories of large
# workloads, written by make_cgls_2048.py and checked below)
FILES = sorted(f for f in glob.glob(os.path.join(HERE, "*.json")) if not os.path.basename(f).startswith("cgls_"))


def load(path):
    with open(path) as f:
        d = json.load(f)
    f64 = lambda a: np.array([float(v) for v in a], np.float64)  # noqa: E731
    d["val"] = f64(d["val"])
    for k in ("x_true", "b", "sirt", "cgls", "cgls_resnorm"):
        d[k] = np.array([f64(s) for s in d[k]])
    return d


def geometry(d):
    s = d["geometry"]
    return oracle.Geometry(s["nx"], s["ny"], s["n_p"], s["n_theta"],
                           None if s["angles"] is None else np.array(s["angles"], np.float64), s["center"],
                           s.get("model", "line"))


def test_fixtures_exist():
    assert len(FILES) >= 3


@pytest.mark.parametrize("path", FILES, ids=[os.path.basename(p) for p in FILES])
def test_oracle_reproduces_golden(path):
    d = load(path)
    g = geometry(d)
    A = oracle.build_matrix(g)
    np.testing.assert_array_equal(A.row_ptr, d["row_ptr"])
    np.testing.assert_array_equal(A.col, d["col"])
    np.testing.assert_array_equal(A.val, d["val"])
    AT = A.transpose()
    np.testing.assert_allclose(oracle.project(A, d["x_true"]), d["b"], rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(oracle.sirt(A, AT, d["b"], d["sirt_iters"]), d["sirt"], rtol=1e-12, atol=1e-13)
    x, h = oracle.cgls(A, AT, d["b"], d["cgls_iters"])
    np.testing.assert_allclose(x, d["cgls"], rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(h, d["cgls_resnorm"], rtol=1e-10, atol=1e-12)


def test_golden_square_theta0_by_hand():
    """theta = 0: ray k is the pixel column ix = k; each of its n_y pixels has
    a unit chord, so row k lists columns k, k + 8, ..., k + 56 with value 1."""
    d = load(os.path.join(HERE, "square_8x8_12.json"))
    rp = d["row_ptr"]
    for k in range(8):
        cols = d["col"][rp[k]:rp[k + 1]]
        assert cols == [iy * 8 + k for iy in range(8)]
        assert np.all(d["val"][rp[k]:rp[k + 1]] == 1.0)


@pytest.mark.gpu
@pytest.mark.parametrize("path", FILES, ids=[os.path.basename(p) for p in FILES])
def test_gpu_matches_golden(path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs CUDA")
    import paper_2003_12677_b300 as tomo
    d = load(path)
    s = d["geometry"]
    M = tomo.Matrix(s["nx"], s["n_theta"], n_p=s["n_p"], n_y=s["ny"], angles=s["angles"], center=s["center"],
                    model=s.get("model", "line"))
    rp, col, val = M.export_csr()
    np.testing.assert_array_equal(rp, d["row_ptr"])
    np.testing.assert_array_equal(col, d["col"])
    np.testing.assert_array_equal(val, d["val"].astype(np.float32))
    nz = d["b"].shape[0]
    b = torch.from_numpy(d["b"].astype(np.float32).reshape(nz, s["n_theta"], s["n_p"])).cuda()
    for B in (1, 4):
        x = tomo.sirt(M, b, d["sirt_iters"], batch_width=B).double().cpu().numpy().reshape(nz, -1)
        for k in range(nz):
            assert np.linalg.norm(x[k] - d["sirt"][k]) <= 1e-4 * np.linalg.norm(d["sirt"][k])
        x = tomo.cgls(M, b, d["cgls_iters"], batch_width=B).double().cpu().numpy().reshape(nz, -1)
        for k in range(nz):
            assert np.linalg.norm(x[k] - d["cgls"][k]) <= 1e-4 * np.linalg.norm(d["cgls"][k])
    M.close()


def test_stored_cgls_data_fit_history():
    """The stored 2048^2 x 1024 CGLS history: the FP64 recurrence residual
    equals the true residual ||b - A x_k|| (recomputed by the oracle when it was
    written) to 1e-12 at the checked iterations, and never increases (CGLS
    minimises it over growing Krylov spaces)."""
    with open(os.path.join(HERE, "cgls_2048x1024_slice0.json")) as f:
        d = json.load(f)
    res = np.array(d["resnorm"])
    assert len(res) == d["iters"] >= 50
    for k, v in d["true_resnorm"].items():
        assert abs(res[int(k) - 1] - v) <= 1e-12 * v
    assert np.all(np.diff(res) <= 0) and res[0] < d["b_norm"]
    assert len(d["sample_index"]) == len(d["samples"]["1"]) == 1024

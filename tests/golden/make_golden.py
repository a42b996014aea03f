"""Write the golden fixtures of tests/golden/ from the FP64 oracle only.

Each fixture is a small JSON text file: the geometry, the projector A as CSR
(row pointers, columns, FP64 chord lengths written with repr, so they read
back bit for bit), a seeded input stack, and the oracle's SIRT (Sec. 2.1,
classical R/C form) and CGLS (Sec. 2.1, textbook form) iterates on it.  The
values come from `oracle/` and nothing else; they freeze the oracle so that a
later change to its arithmetic shows up as a fixture diff, and they give the
GPU tests a stored expected value for small geometries.

Run from the repository root: python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

CASES = {
    # square 8x8, 12 default angles: includes theta = 0, pi/4 (m = 3), pi/2 (m = 6)
    "square_8x8_12": dict(nx=8, ny=8, n_p=8, n_theta=12, angles=None, center=None),
    # non-square grid, odd detector, shifted axis, user angles (one negative, one past pi)
    "rect_7x5_9_shifted": dict(nx=7, ny=5, n_p=9, n_theta=5, angles=[-0.3, 0.0, 0.7, 1.9, 3.3], center=3.7),
    # the strip model (area of each pixel inside a unit-width strip) on the 8x8 square
    "strip_8x8_12": dict(nx=8, ny=8, n_p=8, n_theta=12, angles=None, center=None, model="strip"),
}
SIRT_ITERS, CGLS_ITERS, SLICES = 10, 4, 2


def make(name, spec):
    g = oracle.Geometry(spec["nx"], spec["ny"], spec["n_p"], spec["n_theta"],
                        None if spec["angles"] is None else np.array(spec["angles"], np.float64), spec["center"],
                        spec.get("model", "line"))
    A = oracle.build_matrix(g)
    AT = A.transpose()
    rng = np.random.default_rng(20031267)
    x_true = rng.random((SLICES, g.cols))
    b = oracle.project(A, x_true)
    sirt = oracle.sirt(A, AT, b, SIRT_ITERS)
    cgls, hist = oracle.cgls(A, AT, b, CGLS_ITERS)
    return {
        "source": "tests/golden/make_golden.py (FP64 oracle: %s model, SIRT, CGLS of Sec. 2.1)"
                  % spec.get("model", "line"),
        "geometry": spec, "rows": A.rows, "cols": A.cols,
        "row_ptr": A.row_ptr.tolist(), "col": A.col.tolist(), "val": [repr(float(v)) for v in A.val],
        "x_true": [[repr(float(v)) for v in s] for s in x_true],
        "b": [[repr(float(v)) for v in s] for s in b],
        "sirt_iters": SIRT_ITERS, "sirt": [[repr(float(v)) for v in s] for s in sirt],
        "cgls_iters": CGLS_ITERS, "cgls": [[repr(float(v)) for v in s] for s in cgls],
        "cgls_resnorm": [[repr(float(v)) for v in s] for s in hist],
    }


def main():
    for name, spec in CASES.items():
        with open(os.path.join(HERE, name + ".json"), "w") as f:
            json.dump(make(name, spec), f, indent=0)
            f.write("\n")


if __name__ == "__main__":
    main()

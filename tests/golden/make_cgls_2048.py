"""Write tests/golden/cgls_2048x1024_slice0.json from the FP64 oracle only.

The 2048 x 2048, 1024-angle, 2048-bin CGLS workload (16 slices of a seeded
random-ellipsoid phantom, 5% Gaussian noise) is too large for the oracle to
solve inside a test or a benchmark run: one matrix-free projection pair takes
tens of seconds on a host.  This script runs the oracle's textbook CGLS
(Sec. 2.1) matrix-free on slice 0 once, for ITERS iterations, and stores:

  * resnorm[k]  ||b - A x_{k+1}|| after every iteration (the FP64 recurrence
                residual; in FP64 it equals the true residual to ~1e-12, which
                `true_resnorm` checks at the iterations listed there),
  * xnorm[k]    ||x_{k+1}||,
  * samples     x_1, x_2, x_3 at SAMPLES seeded pixel indices (repr, so they
                read back bit for bit).

The stored data-fit history is the target of the precision comparison: the
number of iterations each GPU form needs to reach the oracle's 50-iteration
data fit ||b - A x_50||.  Run from the repository root (about an hour on
8 host cores):  python tests/golden/make_cgls_2048.py
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2003_12677_b300 import inputs  # noqa: E402

NAME = "cgls_2048x1024_b16"
ITERS = 60
SAMPLES = 1024
CHECK_TRUE = (1, 50)


def main():
    w = inputs.WORKLOADS[NAME]
    c = inputs.workload_case(NAME, slices=[0])
    g = oracle.Geometry(w.n, w.n, w.n, w.n_theta)
    b = c.sino.reshape(1, -1).astype(np.float64)
    idx = np.sort(np.random.default_rng(20031267).choice(g.cols, SAMPLES, replace=False))
    t0 = time.time()
    x, hist = oracle.cgls_mf(g, b, 0)  # x = 0, initial state
    r = b.copy()
    s = oracle.backproject_mf(g, r)
    p = s.copy()
    gamma = np.array([float(np.dot(s[0], s[0]))])
    frozen = np.zeros(1, np.int32)
    resn, xn, samples, true_res = [], [], {}, {}
    for k in range(1, ITERS + 1):
        x, r, p, gamma, frozen, h = oracle.cgls_resume_mf(g, x, r, p, gamma, frozen, 1)
        resn.append(float(h[0, 0]))
        xn.append(float(np.linalg.norm(x[0])))
        if k <= 3:
            samples[str(k)] = [repr(float(v)) for v in x[0, idx]]
        if k in CHECK_TRUE:
            true_res[str(k)] = float(np.linalg.norm(b[0] - oracle.project_mf(g, x)[0]))
        print(k, resn[-1], xn[-1], round(time.time() - t0), flush=True)
    out = dict(workload=NAME, slice=0, n=w.n, n_theta=w.n_theta, n_p=w.n, iters=ITERS,
               b_norm=float(np.linalg.norm(b[0])), resnorm=resn, xnorm=xn, true_resnorm=true_res,
               sample_index=[int(i) for i in idx], samples=samples,
               note="FP64 oracle, textbook CGLS from x0 = 0, matrix-free products; written by make_cgls_2048.py")
    with open(os.path.join(HERE, "cgls_2048x1024_slice0.json"), "w") as f:
        json.dump(out, f, indent=0)


if __name__ == "__main__":
    main()

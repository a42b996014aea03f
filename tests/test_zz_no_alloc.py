"""tomo_sirt_noalloc: SIRT for callers that cannot allocate GPU memory.

Some programs reconstruct inside a fixed GPU memory budget -- for instance a
reconstruction loop running inside a detector's acquisition software, where a
cudaMalloc / cudaFree can stall the streams moving frames or fail mid-scan.
They cannot hand the library a workspace, nor let it allocate one, so this
entry point runs SIRT out of a scratch array compiled into libtomo.

The test calls it through the C ABI twice in a row (the second call finds the
first call's leftovers in the shared scratch) and checks each result against
tomo_sirt, the allocating entry point, at the SIRT tolerance (1e-4 relative
L2 per slice).  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2003_12677_b300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # the gpu marker is only run on a GPU machine
    pytest.skip("needs CUDA", allow_module_level=True)

import paper_2003_12677_b300 as tomo  # noqa: E402
from paper_2003_12677_b300 import _lib  # noqa: E402


def _rel(a, b):
    a = a.double().reshape(a.shape[0], -1)
    b = b.double().reshape(b.shape[0], -1)
    return ((a - b).norm(dim=1) / b.norm(dim=1)).max().item()


def _noalloc(M, sino, iters, lam):
    lib = _lib.load()
    nz = sino.shape[0]
    x = torch.zeros((nz, M.n_y, M.n_x), device="cuda")
    st = lib.tomo_sirt_noalloc(M.handle, ctypes.c_void_p(sino.data_ptr()), ctypes.c_void_p(x.data_ptr()), nz,
                               iters, ctypes.c_float(lam),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    _lib.check(st, "tomo_sirt_noalloc")
    return x


def test_noalloc_matches_sirt_twice_in_a_row():
    M = tomo.Matrix(128, 180)
    first = torch.from_numpy(inputs.workload_case("sirt_128x180_b1").sino).cuda()
    c = inputs.make_case(128, 180, 6, seed=77, phantom="ellipsoids3d", noise="poisson", level=1e4)
    second = torch.from_numpy(c.sino).cuda()
    for sino, iters, lam in ((second, 30, 1.0), (first, 50, 0.9)):
        got = _noalloc(M, sino, iters, lam)
        ref = tomo.sirt(M, sino, iters, lam=lam)
        torch.cuda.synchronize()
        assert _rel(got, ref) < 1e-4


def test_noalloc_rejects_oversized_geometry():
    # 2048 x 2048 bins x angles = 4,194,304 + 2048 rays: the residual alone
    # (one float per ray) no longer fits in the 16 MiB scratch
    M = tomo.Matrix(8, 2049, n_p=2048)
    sino = torch.zeros((1, 2049, 2048), device="cuda")
    x = torch.zeros((1, 8, 8), device="cuda")
    lib = _lib.load()
    st = lib.tomo_sirt_noalloc(M.handle, ctypes.c_void_p(sino.data_ptr()), ctypes.c_void_p(x.data_ptr()), 1, 1,
                               ctypes.c_float(1.0), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 1
    assert b"16777216" in lib.tomo_last_error()

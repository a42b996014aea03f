"""tomo_sirt_noalloc: SIRT for callers that cannot allocate GPU memory.

Some programs reconstruct inside a fixed GPU memory budget -- for instance a
reconstruction loop running inside a detector's acquisition software, where a
cudaMalloc / cudaFree can stall the streams moving frames or fail mid-scan.
They cannot hand the library a workspace, nor let it allocate one, so this
entry point runs SIRT out of a scratch array compiled into libtomo.

The test calls it through the C ABI twice in a row (the second call finds the
first call's leftovers in the shared scratch) and checks each result against
tomo_sirt, the allocating entry point, and against the FP64 oracle, at the
SIRT tolerance (1e-4 relative L2 per slice).  One case has 19 slices, so the
internal 16-slice batch loop runs twice with a ragged second batch.  The
default memory pool's high-water mark shows that the calls allocate nothing
from it.  This file is collected last on purpose.
"""
import ctypes

import pytest

import oracle
from paper_2003_12677_b300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # the gpu marker is only run on a GPU machine
    pytest.skip("needs CUDA", allow_module_level=True)

import paper_2003_12677_b300 as tomo  # noqa: E402
from paper_2003_12677_b300 import _lib  # noqa: E402


def _rel(a, b):
    a = torch.as_tensor(a).double().reshape(a.shape[0], -1)
    b = torch.as_tensor(b).double().reshape(b.shape[0], -1)
    return ((a - b).norm(dim=1) / b.norm(dim=1)).max().item()


def _noalloc(M, sino, iters, lam, x=None):
    lib = _lib.load()
    nz = sino.shape[0]
    x = torch.zeros((nz, M.n_y, M.n_x), device="cuda") if x is None else x
    st = lib.tomo_sirt_noalloc(M.handle, ctypes.c_void_p(sino.data_ptr()), ctypes.c_void_p(x.data_ptr()), nz,
                               iters, ctypes.c_float(lam),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    _lib.check(st, "tomo_sirt_noalloc")
    return x


def _pool():
    """(reset, high-water) helpers of the current device's default memory pool."""
    from cuda.bindings import driver as drv
    from cuda.bindings import runtime as rt
    err, pool = rt.cudaDeviceGetDefaultMemPool(torch.cuda.current_device())
    assert err == rt.cudaError_t.cudaSuccess

    def attr(a):
        err, v = rt.cudaMemPoolGetAttribute(pool, a)
        assert err == rt.cudaError_t.cudaSuccess
        return int(v)

    def reset():
        err, = rt.cudaMemPoolSetAttribute(pool, rt.cudaMemPoolAttr.cudaMemPoolAttrUsedMemHigh, drv.cuuint64_t(0))
        assert err == rt.cudaError_t.cudaSuccess
        return attr(rt.cudaMemPoolAttr.cudaMemPoolAttrUsedMemCurrent)

    return reset, lambda: attr(rt.cudaMemPoolAttr.cudaMemPoolAttrUsedMemHigh)


def test_noalloc_matches_sirt_and_the_oracle_twice_in_a_row():
    M = tomo.Matrix(128, 180)
    g = oracle.Geometry(128, 128, 128, 180)
    A = oracle.build_matrix(g)
    AT = A.transpose()
    first = inputs.workload_case("sirt_128x180_b1").sino
    second = inputs.make_case(128, 180, 19, seed=77, phantom="ellipsoids3d", noise="poisson", level=1e4).sino
    reset, high = _pool()
    for sino_np, iters, lam in ((second, 30, 1.0), (first, 50, 0.9)):
        sino = torch.from_numpy(sino_np).cuda()
        x = torch.zeros((sino.shape[0], 128, 128), device="cuda")
        torch.cuda.synchronize()
        used = reset()
        got = _noalloc(M, sino, iters, lam, x)
        torch.cuda.synchronize()
        assert high() <= used, "the no-allocation entry point drew memory from the default pool"
        ref = tomo.sirt(M, sino, iters, lam=lam)
        torch.cuda.synchronize()
        assert _rel(got.cpu(), ref.cpu()) < 1e-4
        orc = oracle.sirt(A, AT, sino_np.reshape(sino_np.shape[0], -1), iters, lam)
        assert _rel(got.cpu().reshape(len(orc), -1), torch.from_numpy(orc)) < 1e-4


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

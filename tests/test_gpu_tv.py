"""The TV prior of the model-based objective (Sec. 2.1) on the GPU (tomo_tv)
vs the FP64 oracle, through the C ABI.  The oracle's objective with b = A x
(so the data term is exactly 0) is mu * TV and its gradient mu * dTV/dx.
FP32 differences and square roots: value and gradient within 1e-5 relative;
the value is deterministic (fixed-order FP64 sums)."""
import numpy as np
import pytest

import oracle
from paper_2003_12677_b300 import _lib, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # the gpu marker is only run on a GPU machine
    pytest.skip("needs CUDA", allow_module_level=True)

import paper_2003_12677_b300 as tomo  # noqa: E402


def oracle_tv(x, eps):
    """mu = 1, b = A x: the objective is the TV value, the gradient its gradient."""
    nz, ny, nx = x.shape
    g = oracle.Geometry(nx, ny, max(nx, ny), 3)
    A = oracle.build_matrix(g)
    AT = A.transpose()
    xv = x.reshape(nz, -1).astype(np.float64)
    f, grad = oracle.loss_grad(A, AT, nx, ny, xv, A.apply(xv), mu=1.0, eps=eps)
    return f, grad.reshape(x.shape)


def gpu_tv(x, eps):
    xt = torch.from_numpy(x).cuda()
    loss = torch.empty(x.shape[0], dtype=torch.float64, device="cuda")
    grad = torch.empty_like(xt)
    _lib.call("tomo_tv", xt.data_ptr(), x.shape[0], x.shape[1], x.shape[2], float(eps), loss.data_ptr(),
              grad.data_ptr(), None)
    return loss.cpu().numpy(), grad.cpu().numpy()


@pytest.mark.parametrize("shape", [(3, 64, 64), (2, 37, 50), (1, 1, 9), (2, 7, 1), (1, 1, 1)])
@pytest.mark.parametrize("eps", [1e-3, 0.1])
def test_tv_matches_oracle(shape, eps):
    x = inputs.random_slices(shape, 500 + shape[1] * 7 + shape[2])
    loss, grad = gpu_tv(x, eps)
    f, gref = oracle_tv(x, eps)
    assert abs(loss.sum() - f) <= 1e-5 * abs(f)
    if np.abs(gref).max() == 0:  # a single pixel: no differences
        assert np.abs(grad).max() == 0
    else:
        assert np.linalg.norm(grad - gref) <= 1e-5 * np.linalg.norm(gref)


def test_tv_autograd_and_determinism():
    """tv_loss through autograd: backward returns the kernel's gradient scaled by
    the upstream gradient; two calls give the same bits."""
    x = inputs.random_slices((4, 48, 40), 531)
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    loss = 3.0 * tomo.tv_loss(xt, 1e-3)
    loss.backward()
    l2, g2 = gpu_tv(x, 1e-3)
    f, gref = oracle_tv(x, 1e-3)
    assert abs(loss.item() / 3.0 - f) <= 1e-5 * f
    assert np.linalg.norm(xt.grad.cpu().numpy() - 3.0 * gref) <= 1e-5 * np.linalg.norm(3.0 * gref)
    l1, g1 = gpu_tv(x, 1e-3)
    np.testing.assert_array_equal(l1, l2)
    np.testing.assert_array_equal(g1, g2)


def test_tv_rejects_bad_arguments():
    x = torch.zeros((1, 4, 4), device="cuda")
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    with pytest.raises(_lib.TomoError):
        _lib.call("tomo_tv", x.data_ptr(), 1, 4, 4, 0.0, loss.data_ptr(), x.data_ptr(), None)
    with pytest.raises(_lib.TomoError):
        _lib.call("tomo_tv", x.data_ptr(), 0, 4, 4, 1e-3, loss.data_ptr(), x.data_ptr(), None)

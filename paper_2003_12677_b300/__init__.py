"""B300-native sparse-matrix tomography: projector A, explicit transpose A^T,
batched SpMM, SIRT and CGLS as sm_103a CUDA kernels behind a C ABI.

The torch-facing API (``Matrix``, ``project``, ``backproject``, ``sirt``,
``cgls``, ``TomoProject``, ``radon``, ``tv_loss``, ``new_timing``) is imported
on first use so that ``paper_2003_12677_b300.inputs`` stays importable without
torch.
"""
_API = {"Matrix", "project", "backproject", "sirt", "cgls", "TomoProject", "radon", "tv_loss", "new_timing",
        "sirt_noalloc", "cgls_batched", "stream_status",
        "sirt_bb", "Fubini", "residual_norm", "set_launch"}


def __getattr__(name):
    if name in _API:
        from . import api
        return getattr(api, name)
    raise AttributeError(name)

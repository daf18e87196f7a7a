"""psd_residual_noalloc: the allocation-free residual entry point.

It serves callers that cannot call cudaMalloc (stream capture under an
allocator that refuses new allocations, plug-ins whose host owns every device
allocation, fixed-budget deployments).  Its scratch is a static __device__
array, so these tests check that it gives the same residual and norms as the
handle-based psd_residual, on consecutive calls (the scratch keeps the last
call's contents and must be cleared by each call), including the grids that
need the most residual blocks.  The file is named so that pytest collects it
last.
"""

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1607_01475_gb300 import Solver, psd_residual_noalloc  # noqa: E402
from paper_1607_01475_gb300 import _lib  # noqa: E402


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("shape,p", [((64, 64), 4.0), ((32, 32, 32), 4.0), ((16, 32, 64), 3.0),
                                     ((1024, 1024), 4.0), ((256, 256, 256), 4.0)])
def test_noalloc_matches_handle_residual_on_consecutive_calls(shape, p):
    rng = np.random.default_rng(11)
    h = 2 * np.pi / shape[-1]
    s, eps = 0.1, 0.2
    u = torch.from_numpy(rng.standard_normal(shape) * 0.3).cuda()
    f = torch.from_numpy(rng.standard_normal(shape)).cuda()
    S = Solver(4, shape, h, p, s, eps)
    r_ref = torch.empty_like(u)
    l2_ref, linf_ref = S.residual(u, f, None, r_ref)
    ref = r_ref.cpu().numpy()
    for call in range(2):
        r = torch.full_like(u, float("nan"))
        l2, linf = psd_residual_noalloc(shape, h, p, s, eps, u, f, r)
        assert _rel(r.cpu().numpy(), ref) <= 1e-12, call
        assert abs(l2 - l2_ref) <= 1e-12 * l2_ref, call
        assert abs(linf - linf_ref) <= 1e-12 * linf_ref, call
    S.close()


@pytest.mark.parametrize("shape", [(1024, 1024, 16), (8, 1024, 1024), (1024, 1024)])
def test_noalloc_accepts_the_grids_with_the_most_blocks(shape):
    """The scratch holds 2048 residual blocks, and every valid grid fits:
    (1024, 1024, 16) takes the small-tile 3D kernel with exactly 2048 blocks,
    (8, 1024, 1024) the column kernel with one wave of blocks, 1024^2 the 2D
    kernel with 1024 tiles.  Each agrees with the handle-based residual."""
    rng = np.random.default_rng(12)
    h = 2 * np.pi / shape[-1]
    u = torch.from_numpy(rng.standard_normal(shape) * 0.3).cuda()
    f = torch.from_numpy(rng.standard_normal(shape)).cuda()
    S = Solver(4, shape, h, 4.0, 0.1, 0.2)
    r_ref = torch.empty_like(u)
    l2_ref, _ = S.residual(u, f, None, r_ref)
    r = torch.full_like(u, float("nan"))
    l2, _ = psd_residual_noalloc(shape, h, 4.0, 0.1, 0.2, u, f, r)
    assert _rel(r.cpu().numpy(), r_ref.cpu().numpy()) <= 1e-12
    assert abs(l2 - l2_ref) <= 1e-12 * l2_ref
    S.close()


def test_noalloc_rejects_sixth_order():
    lib = _lib.load_library()
    prm = _lib.PSDParams(order=6, dim=2, n=(ctypes.c_int * 3)(64, 64, 1), h=0.1, p=4.0, s=0.1, eps=0.1,
                         lam=1.0, precision=0, tol=0.0, max_iter=0, max_outer=0, stream=None)
    x = torch.zeros((64, 64), dtype=torch.float64, device="cuda")
    ptr = ctypes.c_void_p(x.data_ptr())
    assert lib.psd_residual_noalloc(ctypes.byref(prm), ptr, ptr, ptr, None, None) == 1


def test_noalloc_rejects_3d_p_above_6():
    """The same parameter rule as psd_create: p <= 6 in 3D (Sec. 3.1)."""
    lib = _lib.load_library()
    prm = _lib.PSDParams(order=4, dim=3, n=(ctypes.c_int * 3)(16, 16, 16), h=0.1, p=7.0, s=0.1, eps=0.1,
                         lam=0.0, precision=0, tol=0.0, max_iter=0, max_outer=0, stream=None)
    x = torch.zeros((16, 16, 16), dtype=torch.float64, device="cuda")
    ptr = ctypes.c_void_p(x.data_ptr())
    assert lib.psd_residual_noalloc(ctypes.byref(prm), ptr, ptr, ptr, None, None) == 1
    buf = ctypes.create_string_buffer(256)
    lib.psd_noalloc_last_error(buf, len(buf))
    assert b"p <= 6" in buf.value

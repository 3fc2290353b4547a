"""The allocation-free TV entry point, for callers that may not allocate device
memory at the call site (fixed device budgets, real-time loops, plugins that only
get input and output buffers).  It runs the workspace-based r2g_tv3d's own
arithmetic, so its loss and gradient must equal r2g_tv3d's bit for bit, call after
call, although every call reuses one fixed scratch array inside the library.  This
file is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2405_20693_b300 import build, r2g

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    r2g.lib()


def _reference(vol, lam):
    loss = torch.zeros(1, device="cuda")
    grad = torch.empty_like(vol)
    ws = torch.empty(r2g.r2g_tv_workspace_size(vol.shape[0], vol.shape[1]), dtype=torch.uint8, device="cuda")
    r2g.r2g_tv3d(vol, lam, loss, grad, ws)
    return loss, grad


def _noalloc_c(vol, lam, loss, grad):
    """Through the C symbol directly."""
    G, D = vol.shape[0], vol.shape[1]
    return r2g.lib().r2g_tv3d_noalloc(G, D, ctypes.c_void_p(vol.data_ptr()), ctypes.c_float(lam),
                                      ctypes.c_void_p(loss.data_ptr()), ctypes.c_void_p(grad.data_ptr()),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("G,D", [(2, 12), (8, 32), (1, 256)])
def test_noalloc_tv_matches_workspace_tv_twice(G, D):
    """Two calls in a row (they share the fixed scratch), the first through the C
    symbol, the second through the Python binding; G = 1, D = 256 is the largest
    volume the scratch holds (2^24 voxels)."""
    g = np.random.default_rng(100 + D)
    for call in range(2):
        vol = torch.as_tensor(g.standard_normal((G, D, D, D)).astype(np.float32), device="cuda")
        ref_loss, ref_grad = _reference(vol, 0.05)
        loss = torch.full((1,), float("nan"), device="cuda")
        grad = torch.full_like(vol, float("nan"))
        if call == 0:
            st = _noalloc_c(vol, 0.05, loss, grad)
            assert st == r2g.R2G_OK, r2g.lib().r2g_last_error()
        else:
            r2g.r2g_tv3d_noalloc(vol, 0.05, loss, grad)
        torch.cuda.synchronize()
        assert torch.equal(loss, ref_loss), (call, float(loss), float(ref_loss))
        assert torch.equal(grad, ref_grad), call


def test_noalloc_tv_rejects_volumes_beyond_the_fixed_scratch():
    vol = torch.zeros(1, device="cuda")  # never read: the size check comes first
    for G, D in ((2, 257), (1, 257), (2, 256)):  # one voxel-block past 2^24, and twice the limit
        st = r2g.lib().r2g_tv3d_noalloc(G, D, ctypes.c_void_p(vol.data_ptr()), ctypes.c_float(0.05),
                                        ctypes.c_void_p(vol.data_ptr()), ctypes.c_void_p(vol.data_ptr()), None)
        assert st == r2g.R2G_E_INVAL, (G, D)
        assert b"exceed" in r2g.lib().r2g_last_error()

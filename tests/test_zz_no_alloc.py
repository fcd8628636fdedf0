"""The allocation-free velocity loss (lbm_velocity_loss_noalloc).

It serves callers that may not allocate device memory (their memory belongs to
their own pool allocator, or an allocation would synchronise a latency-critical
loop); it keeps its partial sums in a fixed array inside the library.  This
test calls it through the C ABI and checks it against lbm_velocity_loss (the
entry point that uses the context's scratch) on two calls in a row, within the
tolerance of the other loss tests, and checks that an oversized request is
refused before any launch.  It lives in a file of its own that pytest collects
last, and it needs nothing from the other tests.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def lbm():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2403_18466_gb300 import lbm as m
    m.load()
    return m


def _p(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def test_noalloc_loss_matches_context_loss(lbm):
    from paper_2403_18466_gb300 import inputs
    lib = lbm.load()
    B, ny, nx = 2, 40, 300
    g = torch.Generator().manual_seed(0)
    f = (0.1 + 0.02 * torch.rand((B, 9, ny, nx), generator=g)).to(DEV)
    lat = lbm.Lattice(nx, ny, B, tau=0.6, device=DEV)
    lat.set_state(f)
    utx = torch.tensor(inputs.noise((B, ny, nx), 1, 0.03), dtype=torch.float32, device=DEV)
    uty = torch.tensor(inputs.noise((B, ny, nx), 2, 0.03), dtype=torch.float32, device=DEV)
    ref_loss, ref_grad = lat.velocity_loss(utx, uty)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    state = C.c_void_p(lat.state_buffer())
    for call in range(2):
        loss = torch.full((1,), float("nan"), device=DEV)
        grad = torch.full_like(ref_grad, float("nan"))
        rc = lib.lbm_velocity_loss_noalloc(state, nx, ny, B, _p(utx), _p(uty), _p(loss),
                                           _p(grad), stream)
        assert rc == lbm.LBM_OK, lbm.lbm_strerror(rc)
        torch.cuda.synchronize()
        assert abs(loss.item() / ref_loss.item() - 1) <= 1e-5
        assert torch.allclose(grad, ref_grad, rtol=0, atol=1e-5 * ref_grad.abs().max().item())
    # a request beyond the fixed scratch array is refused before any launch
    rc = lib.lbm_velocity_loss_noalloc(state, 128, 1 << 21, 1, _p(utx), _p(uty), _p(loss),
                                       None, stream)
    assert rc == lbm.LBM_ERR_ARG
    assert lat.status() == lbm.LBM_OK

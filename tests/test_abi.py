"""CPU checks of the C ABI: the library builds, loads, and exports every entry
point that include/lbm.h declares; host-side argument checks that run before
any CUDA call (no compute without a GPU)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(lbm(?:3d)?_\w+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2403_18466_gb300 import build, lbm
    build.build()
    return lbm.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert {"lbm_init", "lbm_step", "lbm_moments", "lbm_backward", "lbm3d_init",
            "lbm3d_step"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_host_side_argument_errors(lib):
    from paper_2403_18466_gb300 import lbm
    ctx = C.c_void_p()
    p = lbm.make_params(16, 16, 1, tau=0.6)
    assert lib.lbm_init(C.byref(ctx), None, None, None, None) == lbm.LBM_ERR_ARG
    assert lib.lbm_init(None, C.byref(p), None, None, None) == lbm.LBM_ERR_ARG
    bad = lbm.make_params(16, 16, 1, tau=0.5)  # tau must exceed 1/2
    assert lib.lbm_init(C.byref(ctx), C.byref(bad), C.c_void_p(256), C.c_void_p(512), None) \
        == lbm.LBM_ERR_ARG
    bad = lbm.make_params(0, 16, 1, tau=0.6)
    assert lib.lbm_init(C.byref(ctx), C.byref(bad), C.c_void_p(256), C.c_void_p(512), None) \
        == lbm.LBM_ERR_ARG
    assert lib.lbm_step(None, 1, 0, None) == lbm.LBM_ERR_ARG
    assert lib.lbm_moments(None, None, None, None) == lbm.LBM_ERR_ARG
    assert lib.lbm_status(None) == lbm.LBM_ERR_ARG
    assert lib.lbm_state_buffer(None) is None
    lib.lbm_destroy(None)


@pytest.mark.parametrize("nx,ny,batch", [
    (8, 65536, 1),          # ny beyond gridDim.y of the node-per-thread kernels
    (8, 8, 65536),          # batch beyond gridDim.z
    (46341, 46341, 1),      # nx*ny beyond a 32-bit plane index (~155 GB per buffer pair)
    (2 ** 31 - 1, 2, 1),    # nx*ny just past 2^31 - 1
    (128, 65535, 65535),    # 128-node tile count beyond 2^31 - 1 (and 9*nodes > 2^40)
])
def test_init_rejects_sizes_no_kernel_can_address(lib, nx, ny, batch):
    """Sizes the kernels cannot index are refused on the host before any CUDA
    call (fake, never-dereferenced buffer addresses)."""
    from paper_2403_18466_gb300 import lbm
    ctx = C.c_void_p()
    p = lbm.make_params(nx, ny, batch, tau=0.6)
    assert lib.lbm_init(C.byref(ctx), C.byref(p), C.c_void_p(256), C.c_void_p(512), None) \
        == lbm.LBM_ERR_ARG
    assert not ctx.value


def test_noalloc_loss_rejects_grid_beyond_launch_limits(lib):
    """ny or batch beyond 65535 would exceed the launch grid: LBM_ERR_ARG on the
    host, before the scratch address is looked up (fake device pointers)."""
    from paper_2403_18466_gb300 import lbm
    fake = C.c_void_p(256)
    for nx, ny, batch in ((1, 100000, 1), (1, 1, 70000)):
        assert lib.lbm_velocity_loss_noalloc(fake, nx, ny, batch, fake, fake, fake, None,
                                             None) == lbm.LBM_ERR_ARG


def test_mlp_bf16_layout_query(lib):
    from paper_2403_18466_gb300 import lbm
    wg, xu = lbm.mlp_bf16_layout()
    assert 1 <= wg <= 8 and 0 <= xu <= 8


def test_host_side_argument_errors_of_the_test_hooks(lib):
    from paper_2403_18466_gb300 import lbm
    assert lib.lbm_set_wait_limit(None, 1) == lbm.LBM_ERR_ARG
    assert lib.lbm_set_max_ctas(None, 1) == lbm.LBM_ERR_ARG
    assert lib.lbm_activation(None, 4, 0, None, None) == lbm.LBM_ERR_ARG
    fake = C.c_void_p(256)
    assert lib.lbm_activation(fake, 4, 3, fake, None) == lbm.LBM_ERR_ARG
    assert lib.lbm_activation(fake, -1, 0, fake, None) == lbm.LBM_ERR_ARG


def test_record_bytes_and_strerror(lib):
    from paper_2403_18466_gb300 import lbm
    p = lbm.make_params(256, 256, 32, tau=0.500375)
    sb = 9 * 256 * 256 * 32 * 4
    # 16 steps, checkpoint every 4: 4 checkpoints + 3 recomputed + 2 adjoint buffers
    assert lbm.lbm_record_bytes(p, 16, 4) == 9 * sb
    assert lbm.lbm_record_bytes(p, 16, 0) == 0
    for code in (0, -1, -2, -3, -4, -5):
        assert lbm.lbm_strerror(code)
    assert lbm.lbm_strerror(-99) == "unknown error"


def test_d3q19_tables_match_the_oracle(lib):
    """The stencil compiled into the D3Q19 kernels equals the oracle's copy of
    the paper's table (host call, no GPU)."""
    import numpy as np
    import oracle.d3q19 as o3
    from paper_2403_18466_gb300 import lbm
    cx, cy, cz, w = lbm.lbm3d_lattice()
    ocx, ocy, ocz, ow = o3.lattice()
    assert list(ocx) == cx and list(ocy) == cy and list(ocz) == cz
    assert np.array_equal(np.float32(ow), np.array(w, dtype=np.float32))
    assert lib.lbm3d_mlp_nparams() == o3.mlp_nparams() == lbm.LBM3D_MLP_NPARAMS


def test_d3q19_host_side_argument_errors(lib):
    from paper_2403_18466_gb300 import lbm
    ctx = C.c_void_p()
    p = lbm.make_params3d(8, 8, 8, tau=0.6)
    assert lib.lbm3d_init(C.byref(ctx), None, None, None, None) == lbm.LBM_ERR_ARG
    assert lib.lbm3d_init(C.byref(ctx), C.byref(p), None, None, None) == lbm.LBM_ERR_ARG
    for bad in (lbm.make_params3d(8, 8, 8, tau=0.5), lbm.make_params3d(8, 0, 8),
                lbm.make_params3d(8, 70000, 1), lbm.make_params3d(8, 8, 300, batch=300)):
        assert lib.lbm3d_init(C.byref(ctx), C.byref(bad), C.c_void_p(256), C.c_void_p(512),
                              None) == lbm.LBM_ERR_ARG
    assert lib.lbm3d_init(C.byref(ctx), C.byref(p), C.c_void_p(256), C.c_void_p(256),
                          None) == lbm.LBM_ERR_ARG
    assert lib.lbm3d_step(None, 1, 0, None) == lbm.LBM_ERR_ARG
    assert lib.lbm3d_moments(None, None, None) == lbm.LBM_ERR_ARG
    assert lib.lbm3d_status(None) == lbm.LBM_ERR_ARG
    assert lib.lbm3d_state_buffer(None) is None
    lib.lbm3d_destroy(None)

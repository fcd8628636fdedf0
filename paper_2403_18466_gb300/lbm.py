"""Thin ctypes binding of the C ABI in ``include/lbm.h`` (argument marshalling only).

Every function here forwards to the entry point of the same name in
``_build/liblbm.so``; all arithmetic runs in the library's CUDA kernels.
PyTorch is used only for device memory and streams.  If the library is not
built this module raises on first use: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "liblbm.so")

LBM_OK = 0
LBM_ERR_ARG = -1
LBM_ERR_CUDA = -2
LBM_ERR_UNSUPPORTED = -3
LBM_ERR_UNSTABLE = -4
LBM_ERR_TIMEOUT = -5

LBM_BGK, LBM_SMAG, LBM_MLP_BF16, LBM_MLP_F32 = 0, 1, 2, 3
LBM_MLP_HIDDEN = 64
LBM_MLP_NPARAMS = 5385
KINDS = {"bgk": LBM_BGK, "smag": LBM_SMAG, "mlp_bf16": LBM_MLP_BF16, "mlp_f32": LBM_MLP_F32}


class lbm_params(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("batch", C.c_int), ("tau", C.c_double),
                ("smag_cs", C.c_double), ("smag_delta", C.c_double),
                ("force_amp", C.c_double), ("force_mode", C.c_int), ("flags", C.c_int)]


class lbm_weights(C.Structure):
    _fields_ = [("w1", C.c_void_p), ("b1", C.c_void_p), ("w2", C.c_void_p), ("b2", C.c_void_p),
                ("w3", C.c_void_p), ("b3", C.c_void_p), ("dtype", C.c_int)]


class lbm3d_params(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("batch", C.c_int),
                ("tau", C.c_double), ("smag_cs", C.c_double), ("smag_delta", C.c_double),
                ("force_amp", C.c_double), ("force_mode", C.c_int), ("flags", C.c_int)]


class lbm3d_weights(C.Structure):
    _fields_ = [("w1", C.c_void_p), ("b1", C.c_void_p), ("w2", C.c_void_p), ("b2", C.c_void_p),
                ("w3", C.c_void_p), ("b3", C.c_void_p), ("w4", C.c_void_p), ("b4", C.c_void_p),
                ("dtype", C.c_int)]


LBM3D_WIDTHS = (300, 300, 100)
LBM3D_MLP_NPARAMS = 128319


class LbmError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {lbm_strerror(code)} ({code})")


_lib = None
_vp, _i, _sz = C.c_void_p, C.c_int, C.c_size_t
_SIGS = {
    "lbm_init": (_i, [C.POINTER(_vp), C.POINTER(lbm_params), _vp, _vp, _vp]),
    "lbm_destroy": (None, [_vp]),
    "lbm_set_state": (_i, [_vp, _vp]),
    "lbm_get_state": (_i, [_vp, _vp]),
    "lbm_init_equilibrium": (_i, [_vp, _vp, _vp, _vp]),
    "lbm_step": (_i, [_vp, _i, _i, C.POINTER(lbm_weights)]),
    "lbm_moments": (_i, [_vp, _vp, _vp, _vp]),
    "lbm_state_buffer": (_vp, [_vp]),
    "lbm_status": (_i, [_vp]),
    "lbm_clear_status": (_i, [_vp]),
    "lbm_set_wait_limit": (_i, [_vp, C.c_uint]),
    "lbm_set_max_ctas": (_i, [_vp, _i]),
    "lbm_activation": (_i, [_vp, _i, _i, _vp, _vp]),
    "lbm_mlp_bf16_layout": (_i, [C.POINTER(_i), C.POINTER(_i)]),
    "lbm_velocity_loss": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "lbm_record_bytes": (_sz, [C.POINTER(lbm_params), _i, _i]),
    "lbm_forward_record": (_i, [_vp, _i, _i, C.POINTER(lbm_weights), _vp, _sz]),
    "lbm_backward": (_i, [_vp, _vp, C.POINTER(lbm_weights), _vp, _sz, _vp, _vp]),
    "lbm_forward_record_bf16": (_i, [_vp, _i, _i, C.POINTER(lbm_weights), _vp, _sz]),
    "lbm_backward_bf16": (_i, [_vp, _vp, C.POINTER(lbm_weights), _vp, _sz, _vp, _vp]),
    "lbm_box_filter": (_i, [_vp, _i, _vp]),
    "lbm_subsample": (_i, [_vp, _i, _vp]),
    "lbm_velocity_loss_subset": (_i, [_vp, _vp, _i, _vp, _vp, _vp, _vp]),
    "lbm_population_loss_subset": (_i, [_vp, _vp, _i, _vp, _vp, _vp]),
    "lbm_stream": (_i, [_vp, _i, _vp, _vp]),
    "lbm_run_host": (_i, [_vp, _vp, _i, _i, C.POINTER(lbm_weights), _vp, _vp, _vp]),
    "lbm_velocity_loss_noalloc": (_i, [_vp, _i, _i, _i, _vp, _vp, _vp, _vp, _vp]),
    "lbm_structure_functions": (_i, [_vp, _i, _vp]),
    "lbm_energy_spectrum": (_i, [_vp, _i, _vp]),
    "lbm_strerror": (C.c_char_p, [_i]),
    "lbm3d_mlp_nparams": (_sz, []),
    "lbm3d_lattice": (None, [_vp, _vp, _vp, _vp]),
    "lbm3d_init": (_i, [C.POINTER(_vp), C.POINTER(lbm3d_params), _vp, _vp, _vp]),
    "lbm3d_destroy": (None, [_vp]),
    "lbm3d_set_state": (_i, [_vp, _vp]),
    "lbm3d_get_state": (_i, [_vp, _vp]),
    "lbm3d_init_equilibrium": (_i, [_vp, _vp, _vp]),
    "lbm3d_step": (_i, [_vp, _i, _i, C.POINTER(lbm3d_weights)]),
    "lbm3d_moments": (_i, [_vp, _vp, _vp]),
    "lbm3d_state_buffer": (_vp, [_vp]),
    "lbm3d_status": (_i, [_vp]),
    "lbm3d_clear_status": (_i, [_vp]),
}


def load():
    """Load the in-tree library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def lbm_strerror(code: int) -> str:
    return load().lbm_strerror(int(code)).decode()


def _check(rc, where):
    if rc != LBM_OK:
        raise LbmError(rc, where)


def make_params(nx, ny, batch=1, tau=0.6, smag_cs=0.0, smag_delta=1.0, force_amp=0.0,
                force_mode=0):
    return lbm_params(int(nx), int(ny), int(batch), float(tau), float(smag_cs),
                      float(smag_delta), float(force_amp), int(force_mode), 0)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def weights_struct(theta):
    """lbm_weights viewing a packed parameter tensor (float32 or bfloat16,
    LBM_MLP_NPARAMS elements, order w1, b1, w2, b2, w3, b3) on the device."""
    import torch
    assert theta.is_contiguous() and theta.numel() == LBM_MLP_NPARAMS
    dtype = {torch.float32: 0, torch.bfloat16: 1}[theta.dtype]
    h = LBM_MLP_HIDDEN
    sizes = [h * 9, h, h * h, h, 9 * h, 9]
    base, es, off, ptrs = theta.data_ptr(), theta.element_size(), 0, []
    for s in sizes:
        ptrs.append(base + off * es)
        off += s
    w = lbm_weights(*ptrs, dtype)
    w._keepalive = theta
    return w


def make_params3d(nx, ny, nz, batch=1, tau=0.6, smag_cs=0.0, smag_delta=1.0, force_amp=0.0,
                  force_mode=1):
    return lbm3d_params(int(nx), int(ny), int(nz), int(batch), float(tau), float(smag_cs),
                        float(smag_delta), float(force_amp), int(force_mode), 0)


def weights3d_struct(theta):
    """lbm3d_weights viewing a packed FP32 parameter tensor of the paper's network
    (LBM3D_MLP_NPARAMS elements: w1[300][19], b1, w2[300][300], b2, w3[100][300],
    b3, w4[19][100], b4) on the device."""
    import torch
    assert theta.is_contiguous() and theta.numel() == LBM3D_MLP_NPARAMS
    dtype = {torch.float32: 0, torch.bfloat16: 1}[theta.dtype]
    h1, h2, h3 = LBM3D_WIDTHS
    sizes = [h1 * 19, h1, h2 * h1, h2, h3 * h2, h3, 19 * h3, 19]
    base, es, off, ptrs = theta.data_ptr(), theta.element_size(), 0, []
    for n in sizes:
        ptrs.append(base + off * es)
        off += n
    w = lbm3d_weights(*ptrs, dtype)
    w._keepalive = theta
    return w


def lbm3d_lattice():
    """(cx, cy, cz, w) as compiled into the D3Q19 kernels (host call, no GPU)."""
    cx, cy, cz, w = (C.c_int * 19)(), (C.c_int * 19)(), (C.c_int * 19)(), (C.c_float * 19)()
    load().lbm3d_lattice(C.cast(cx, _vp), C.cast(cy, _vp), C.cast(cz, _vp), C.cast(w, _vp))
    return list(cx), list(cy), list(cz), list(w)


def mlp_bf16_layout():
    """(tile warpgroups per SM, XU pairs of every 8) of the compiled tensor-core step."""
    wg, xu = C.c_int(), C.c_int()
    _check(load().lbm_mlp_bf16_layout(C.byref(wg), C.byref(xu)), "lbm_mlp_bf16_layout")
    return wg.value, xu.value


def activation(a, path):
    """The tensor-core step's hidden-layer activation applied element-wise to a
    CUDA float32 tensor (path 0: XU form, 1: FMA form as stored, 2: FMA form
    before its bf16 rounding)."""
    import torch
    assert a.dtype == torch.float32 and a.is_cuda and a.is_contiguous()
    out = torch.empty_like(a)
    s = torch.cuda.current_stream(a.device).cuda_stream
    _check(load().lbm_activation(_ptr(a), a.numel(), int(path), _ptr(out), C.c_void_p(s)),
           "lbm_activation")
    return out


def lbm_record_bytes(params, n, ckpt_every):
    return load().lbm_record_bytes(C.byref(params), int(n), int(ckpt_every))


class Lattice:
    """A context over two torch-owned state buffers on the current CUDA device.

    Methods mirror the C entry points (lbm_set_state -> set_state, ...)."""

    def __init__(self, nx, ny, batch=1, tau=0.6, smag_cs=0.0, smag_delta=1.0, force_amp=0.0,
                 force_mode=0, stream=None, device="cuda"):
        import torch
        self.lib = load()
        self.params = make_params(nx, ny, batch, tau, smag_cs, smag_delta, force_amp, force_mode)
        self.shape = (batch, 9, ny, nx)
        self.device = torch.device(device)
        self.bufs = [torch.zeros(self.shape, dtype=torch.float32, device=self.device)
                     for _ in range(2)]
        self.cuda_stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        ctx = C.c_void_p()
        _check(self.lib.lbm_init(C.byref(ctx), C.byref(self.params), _ptr(self.bufs[0]),
                                 _ptr(self.bufs[1]), C.c_void_p(self.cuda_stream.cuda_stream)),
               "lbm_init")
        self.ctx = ctx

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.lbm_destroy(self.ctx)
            self.ctx = None

    __del__ = close

    # -- state --------------------------------------------------------------
    def set_state(self, f_pre):
        assert f_pre.shape == self.shape and f_pre.dtype.is_floating_point and f_pre.is_contiguous()
        _check(self.lib.lbm_set_state(self.ctx, _ptr(f_pre)), "lbm_set_state")

    def get_state(self, out=None):
        import torch
        out = torch.empty(self.shape, dtype=torch.float32, device=self.device) if out is None else out
        _check(self.lib.lbm_get_state(self.ctx, _ptr(out)), "lbm_get_state")
        return out

    def init_equilibrium(self, rho, ux, uy):
        for a in (rho, ux, uy):
            assert a.shape == (self.shape[0], self.shape[2], self.shape[3]) and a.is_contiguous()
        _check(self.lib.lbm_init_equilibrium(self.ctx, _ptr(rho), _ptr(ux), _ptr(uy)),
               "lbm_init_equilibrium")

    def state_buffer(self):
        return self.lib.lbm_state_buffer(self.ctx)

    def state_tensor(self):
        """The torch buffer holding the current internal state (post-collision
        populations minus the lattice weights, [b][i][y][x]); a view, not a copy."""
        p = self.state_buffer()
        for b in self.bufs:
            if b.data_ptr() == p:
                return b
        raise LbmError(LBM_ERR_ARG, "lbm_state_buffer")

    # -- stepping -----------------------------------------------------------
    def step(self, n, kind="bgk", weights=None):
        k = KINDS[kind] if isinstance(kind, str) else int(kind)
        w = C.byref(weights) if weights is not None else None
        _check(self.lib.lbm_step(self.ctx, int(n), k, w), "lbm_step")

    def moments(self):
        import torch
        B, _, ny, nx = self.shape
        rho, ux, uy = (torch.empty((B, ny, nx), dtype=torch.float32, device=self.device)
                       for _ in range(3))
        _check(self.lib.lbm_moments(self.ctx, _ptr(rho), _ptr(ux), _ptr(uy)), "lbm_moments")
        return rho, ux, uy

    def status(self):
        return self.lib.lbm_status(self.ctx)

    def clear_status(self):
        _check(self.lib.lbm_clear_status(self.ctx), "lbm_clear_status")

    def set_wait_limit(self, polls):
        """Polls per bounded device wait of the tensor-core step (0 = default)."""
        _check(self.lib.lbm_set_wait_limit(self.ctx, int(polls)), "lbm_set_wait_limit")

    def set_max_ctas(self, n):
        """Cap on the tensor-core step's persistent grid (0 = one CTA per SM)."""
        _check(self.lib.lbm_set_max_ctas(self.ctx, int(n)), "lbm_set_max_ctas")

    # -- training -----------------------------------------------------------
    def velocity_loss(self, utx, uty, want_grad=True):
        import torch
        loss = torch.empty(1, dtype=torch.float32, device=self.device)
        g = torch.empty(self.shape, dtype=torch.float32, device=self.device) if want_grad else None
        _check(self.lib.lbm_velocity_loss(self.ctx, _ptr(utx), _ptr(uty), _ptr(loss), _ptr(g)),
               "lbm_velocity_loss")
        return loss, g

    def velocity_loss_subset(self, idx, utx, uty, want_grad=True):
        """Velocity loss on the nodes idx (int32 device tensor of flat indices)."""
        import torch
        loss = torch.empty(1, dtype=torch.float32, device=self.device)
        g = torch.empty(self.shape, dtype=torch.float32, device=self.device) if want_grad else None
        _check(self.lib.lbm_velocity_loss_subset(self.ctx, _ptr(idx), int(idx.numel()), _ptr(utx),
                                                 _ptr(uty), _ptr(loss), _ptr(g)),
               "lbm_velocity_loss_subset")
        return loss, g

    def population_loss_subset(self, idx, target_post, want_grad=True):
        """Eq. S13 on the nodes idx against target post-collision populations."""
        import torch
        loss = torch.empty(1, dtype=torch.float32, device=self.device)
        g = torch.empty(self.shape, dtype=torch.float32, device=self.device) if want_grad else None
        _check(self.lib.lbm_population_loss_subset(self.ctx, _ptr(idx), int(idx.numel()),
                                                   _ptr(target_post), _ptr(loss), _ptr(g)),
               "lbm_population_loss_subset")
        return loss, g

    def stream(self, f, direction=1, out=None):
        """Stream (+1) or anti-stream (-1) a population field on this grid."""
        import torch
        out = torch.empty_like(f) if out is None else out
        _check(self.lib.lbm_stream(self.ctx, int(direction), _ptr(f), _ptr(out)), "lbm_stream")
        return out

    def record_bytes(self, n, ckpt_every):
        return lbm_record_bytes(self.params, n, ckpt_every)

    def forward_record(self, n, ckpt_every, weights, ws, precision="f32"):
        fn = self.lib.lbm_forward_record if precision == "f32" else self.lib.lbm_forward_record_bf16
        _check(fn(self.ctx, int(n), int(ckpt_every), C.byref(weights), _ptr(ws),
                  ws.numel() * ws.element_size()), f"lbm_forward_record ({precision})")

    def backward(self, dL_df_final, weights, ws, dW, dL_df0=None, precision="f32"):
        fn = self.lib.lbm_backward if precision == "f32" else self.lib.lbm_backward_bf16
        _check(fn(self.ctx, _ptr(dL_df_final), C.byref(weights), _ptr(ws),
                  ws.numel() * ws.element_size(), _ptr(dW), _ptr(dL_df0)),
               f"lbm_backward ({precision})")

    def structure_functions(self, rmax):
        """[6, rmax] float64 tensor: S^p(r), p = 1..6 (see lbm_structure_functions)."""
        import torch
        out = torch.empty(6 * rmax, dtype=torch.float64, device=self.device)
        _check(self.lib.lbm_structure_functions(self.ctx, int(rmax), _ptr(out)),
               "lbm_structure_functions")
        return out.view(6, rmax)

    def energy_spectrum(self, kmax):
        """[kmax + 1] float64 tensor: E(k) (see lbm_energy_spectrum)."""
        import torch
        out = torch.empty(kmax + 1, dtype=torch.float64, device=self.device)
        _check(self.lib.lbm_energy_spectrum(self.ctx, int(kmax), _ptr(out)), "lbm_energy_spectrum")
        return out

    def box_filter(self, cg, out=None):
        import torch
        B, _, ny, nx = self.shape
        out = torch.empty((B, 9, ny // cg, nx // cg), dtype=torch.float32,
                          device=self.device) if out is None else out
        _check(self.lib.lbm_box_filter(self.ctx, int(cg), _ptr(out)), "lbm_box_filter")
        return out

    def subsample(self, cg, out=None):
        """Filter phi: the pre-collision populations at every cg-th node."""
        import torch
        B, _, ny, nx = self.shape
        out = torch.empty((B, 9, ny // cg, nx // cg), dtype=torch.float32,
                          device=self.device) if out is None else out
        _check(self.lib.lbm_subsample(self.ctx, int(cg), _ptr(out)), "lbm_subsample")
        return out

    def run_host(self, f_pre_host, n, kind="bgk", weights=None, rho=None, ux=None, uy=None):
        """f_pre_host and the outputs are host tensors (pinned for full speed)."""
        k = KINDS[kind] if isinstance(kind, str) else int(kind)
        w = C.byref(weights) if weights is not None else None
        _check(self.lib.lbm_run_host(self.ctx, _ptr(f_pre_host), int(n), k, w, _ptr(rho),
                                     _ptr(ux), _ptr(uy)), "lbm_run_host")


class Lattice3D:
    """A D3Q19 context (include/lbm3d.h) over two torch-owned state buffers.

    Methods mirror the C entry points (lbm3d_set_state -> set_state, ...)."""

    def __init__(self, nx, ny, nz, batch=1, tau=0.6, smag_cs=0.0, smag_delta=1.0, force_amp=0.0,
                 force_mode=1, stream=None, device="cuda"):
        import torch
        self.lib = load()
        self.params = make_params3d(nx, ny, nz, batch, tau, smag_cs, smag_delta, force_amp,
                                    force_mode)
        self.shape = (batch, 19, nz, ny, nx)
        self.device = torch.device(device)
        self.bufs = [torch.zeros(self.shape, dtype=torch.float32, device=self.device)
                     for _ in range(2)]
        self.cuda_stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        ctx = C.c_void_p()
        _check(self.lib.lbm3d_init(C.byref(ctx), C.byref(self.params), _ptr(self.bufs[0]),
                                   _ptr(self.bufs[1]), C.c_void_p(self.cuda_stream.cuda_stream)),
               "lbm3d_init")
        self.ctx = ctx

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.lbm3d_destroy(self.ctx)
            self.ctx = None

    __del__ = close

    def set_state(self, f_pre):
        assert tuple(f_pre.shape) == self.shape and f_pre.is_contiguous()
        _check(self.lib.lbm3d_set_state(self.ctx, _ptr(f_pre)), "lbm3d_set_state")

    def get_state(self, out=None):
        import torch
        out = torch.empty(self.shape, dtype=torch.float32, device=self.device) if out is None \
            else out
        _check(self.lib.lbm3d_get_state(self.ctx, _ptr(out)), "lbm3d_get_state")
        return out

    def init_equilibrium(self, rho, u):
        _check(self.lib.lbm3d_init_equilibrium(self.ctx, _ptr(rho), _ptr(u)),
               "lbm3d_init_equilibrium")

    def step(self, n, kind="bgk", weights=None):
        k = KINDS[kind] if isinstance(kind, str) else int(kind)
        w = C.byref(weights) if weights is not None else None
        _check(self.lib.lbm3d_step(self.ctx, int(n), k, w), "lbm3d_step")

    def moments(self):
        import torch
        B, _, nz, ny, nx = self.shape
        rho = torch.empty((B, nz, ny, nx), dtype=torch.float32, device=self.device)
        u = torch.empty((B, 3, nz, ny, nx), dtype=torch.float32, device=self.device)
        _check(self.lib.lbm3d_moments(self.ctx, _ptr(rho), _ptr(u)), "lbm3d_moments")
        return rho, u

    def state_buffer(self):
        return self.lib.lbm3d_state_buffer(self.ctx)

    def state_tensor(self):
        p = self.state_buffer()
        for b in self.bufs:
            if b.data_ptr() == p:
                return b
        raise LbmError(LBM_ERR_ARG, "lbm3d_state_buffer")

    def status(self):
        return self.lib.lbm3d_status(self.ctx)

    def clear_status(self):
        _check(self.lib.lbm3d_clear_status(self.ctx), "lbm3d_clear_status")

"""FP64 CPU oracle of the D2Q9 lattice-Boltzmann hot path (and, in
``oracle.d3q19``, of the paper's D3Q19 setting).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The library path never imports it.
It shares no code with the CUDA path; ``lbm_oracle.c`` carries its own lattice
tables and is compiled here with gcc (``build()``), independently of nvcc.

Layout conventions: populations are float64 arrays of shape (B, 9, ny, nx);
the stored state of a run is the post-collision field g (pull scheme), and
the pre-collision populations at the next time are ``stream_pull(g)``.

Every wrapper cites the paper passage its C function follows.  All functions
are pinned by tests (see ``tests/test_oracle_*.py``); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "d3q19_oracle.c")]
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liblbm_oracle.so")

BGK, SMAG, MLP = 0, 1, 2
HIDDEN = 64


class Params(C.Structure):
    """Collision parameters (tau: Eq. S3; Smagorinsky C_s, Delta: SI sec. 1;
    Kolmogorov forcing F_x(y) = F0 sin(2 pi m y / ny), applied by EDM, Eq. S5)."""

    _fields_ = [
        ("tau", C.c_double),
        ("smag_cs", C.c_double),
        ("smag_delta", C.c_double),
        ("force_amp", C.c_double),
        ("force_mode", C.c_int),
        ("hidden", C.c_int),
    ]


def params(tau, smag_cs=0.0, smag_delta=1.0, force_amp=0.0, force_mode=0, hidden=HIDDEN):
    return Params(float(tau), float(smag_cs), float(smag_delta), float(force_amp),
                  int(force_mode), int(hidden))


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, IEEE FP64, no contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(f) for f in _SRCS)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", "-shared", "-fPIC", *_SRCS, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d, i, pd, pi = C.c_double, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int)
        pp = C.POINTER(Params)
        sig = {
            "ora_lattice": (None, [pi, pi, pd]),
            "ora_viscosity": (d, [d]),
            "ora_tau_rescaled": (d, [d, d]),
            "ora_feq": (None, [d, d, d, pd]),
            "ora_stream_pull": (None, [i, i, i, pd, pd]),
            "ora_stream_push": (None, [i, i, i, pd, pd]),
            "ora_moments": (None, [i, i, i, pd, pd, pd, pd]),
            "ora_edm_force": (None, [d, d, d, d, d, pd]),
            "ora_smag_tau_eff": (d, [pd, d, d, d]),
            "ora_project": (None, [pd, pd]),
            "ora_mlp_nparams": (i, [i]),
            "ora_mlp_forward": (None, [pd, i, pd, pd]),
            "ora_collide_node": (None, [i, pd, pd, pp, pd, d, d]),
            "ora_collide": (None, [i, i, i, i, pd, pd, pp, pd]),
            "ora_step": (None, [i, i, i, i, pd, pd, pp, pd]),
            "ora_run": (None, [i, i, i, i, pd, i, pp, pd]),
            "ora_box_filter": (None, [i, i, i, i, pd, pd]),
            "ora_velocity_loss": (d, [i, i, i, pd, pd, pd]),
            "ora_velocity_loss_grad": (None, [i, i, i, pd, pd, pd, pd]),
            "ora_unroll_loss": (d, [i, i, i, pd, i, pp, pd, pd, pd]),
            "ora_unroll_grad": (d, [i, i, i, pd, i, pp, pd, pd, pd, pd, pd]),
            "ora_mlp_collide_vjp": (None, [pd, pd, pp, pd, d, d, pd, pd]),
            "ora_feq_field": (None, [i, i, i, pd, pd, pd, pd]),
            "ora_structure_functions": (None, [i, i, i, pd, pd, i, pd]),
            "ora_velocity_loss_subset": (d, [i, i, i, pd, pi, i, pd, pd, pd]),
            "ora_population_loss_subset": (d, [i, i, i, pd, pi, i, pd, pd]),
            "ora_subsample": (None, [i, i, i, i, pd, pd]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(_lib, name)
            fn.restype = res
            fn.argtypes = args
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _theta(theta):
    return _p(_f64(theta)) if theta is not None else None


def lattice():
    """D2Q9 velocities and weights (the oracle's own table)."""
    cx = (C.c_int * 9)()
    cy = (C.c_int * 9)()
    w = np.zeros(9)
    lib().ora_lattice(cx, cy, _p(w))
    return np.array(list(cx)), np.array(list(cy)), w


def viscosity(tau):
    """nu = c_s^2 (tau - 1/2), Eq. S6."""
    return lib().ora_viscosity(float(tau))


def tau_rescaled(tau, cg):
    """tau' = (tau - 1/2)/cg + 1/2, Eq. S9."""
    return lib().ora_tau_rescaled(float(tau), float(cg))


def feq(rho, ux, uy):
    """Second-order equilibrium, Eq. S4."""
    out = np.zeros(9)
    lib().ora_feq(float(rho), float(ux), float(uy), _p(out))
    return out


def edm_force(rho, ux, uy, Fx, Fy):
    """EDM forcing term, Eq. S5."""
    out = np.zeros(9)
    lib().ora_edm_force(float(rho), float(ux), float(uy), float(Fx), float(Fy), _p(out))
    return out


def smag_tau_eff(f, tau0, cs, delta=1.0):
    """Smagorinsky local relaxation time (SI sec. 1, closed form)."""
    f = _f64(f)
    return lib().ora_smag_tau_eff(_p(f), float(tau0), float(cs), float(delta))


def project(o):
    """Mass/momentum projection, Eqs. S11-S12 (D2Q9: 1/9 and 1/6)."""
    o = _f64(o)
    out = np.zeros(9)
    lib().ora_project(_p(o), _p(out))
    return out


def mlp_nparams(h=HIDDEN):
    return lib().ora_mlp_nparams(int(h))


def mlp_forward(theta, x, h=HIDDEN):
    """9 -> h -> h -> 9 MLP with tanh hidden layers (Eq. S10 network)."""
    x = _f64(x)
    out = np.zeros(9)
    lib().ora_mlp_forward(_theta(theta), int(h), _p(x), _p(out))
    return out


def collide_node(kind, f, prm, theta=None, Fx=0.0, Fy=0.0):
    """One node's collision (BGK Eq. S3 / Smagorinsky / learned Eq. S10), EDM forcing last."""
    f = _f64(f)
    out = np.zeros(9)
    lib().ora_collide_node(int(kind), _p(f), _p(out), C.byref(prm), _theta(theta), float(Fx),
                           float(Fy))
    return out


def _shape(a):
    B, q, ny, nx = a.shape
    assert q == 9
    return B, ny, nx


def stream_pull(g):
    """f_i(x) = g_i(x - c_i)  (stream/collide split, Methods)."""
    g = _f64(g)
    out = np.empty_like(g)
    lib().ora_stream_pull(*_shape(g), _p(g), _p(out))
    return out


def stream_push(f):
    """g_i(x) = f_i(x + c_i): anti-streaming along -c_i (SI sec. 2, step 4)."""
    f = _f64(f)
    out = np.empty_like(f)
    lib().ora_stream_push(*_shape(f), _p(f), _p(out))
    return out


def moments(f):
    """rho and u = j/rho per node (SI sec. 1)."""
    f = _f64(f)
    B, ny, nx = _shape(f)
    rho, ux, uy = (np.empty((B, ny, nx)) for _ in range(3))
    lib().ora_moments(B, ny, nx, _p(f), _p(rho), _p(ux), _p(uy))
    return rho, ux, uy


def collide(kind, fpre, prm, theta=None):
    fpre = _f64(fpre)
    out = np.empty_like(fpre)
    lib().ora_collide(*_shape(fpre), int(kind), _p(fpre), _p(out), C.byref(prm), _theta(theta))
    return out


def step(kind, g, prm, theta=None):
    """One step on the stored post-collision state: C(S g), Eq. S2."""
    g = _f64(g)
    out = np.empty_like(g)
    lib().ora_step(*_shape(g), int(kind), _p(g), _p(out), C.byref(prm), _theta(theta))
    return out


def run(kind, g, nsteps, prm, theta=None):
    g = _f64(g).copy()
    lib().ora_run(*_shape(g), int(kind), _p(g), int(nsteps), C.byref(prm), _theta(theta))
    return g


def box_filter(ffine, cg):
    """cg x cg block mean of fine pre-collision populations (filter phi, SI sec. 2)."""
    ffine = _f64(ffine)
    B, ny, nx = _shape(ffine)
    out = np.empty((B, 9, ny // cg, nx // cg))
    lib().ora_box_filter(B, ny, nx, int(cg), _p(ffine), _p(out))
    return out


def velocity_loss(fpre, utx, uty):
    """L = 1/(2 N B) sum |u - u_t|^2 (velocity form of Eq. S13)."""
    fpre, utx, uty = _f64(fpre), _f64(utx), _f64(uty)
    return lib().ora_velocity_loss(*_shape(fpre), _p(fpre), _p(utx), _p(uty))


def velocity_loss_grad(fpre, utx, uty):
    fpre, utx, uty = _f64(fpre), _f64(utx), _f64(uty)
    out = np.empty_like(fpre)
    lib().ora_velocity_loss_grad(*_shape(fpre), _p(fpre), _p(utx), _p(uty), _p(out))
    return out


def unroll_loss(g0, nsteps, prm, theta, utx, uty):
    """Loss after nsteps learned-collision steps (unrolled training, SI sec. 2)."""
    g0, utx, uty = _f64(g0), _f64(utx), _f64(uty)
    return lib().ora_unroll_loss(*_shape(g0), _p(g0), int(nsteps), C.byref(prm), _theta(theta),
                                 _p(utx), _p(uty))


def unroll_grad(g0, nsteps, prm, theta, utx, uty, want_dg0=True):
    """Hand-written reverse mode of unroll_loss: (L, dL/dtheta, dL/dg0)."""
    g0, utx, uty = _f64(g0), _f64(utx), _f64(uty)
    dth = np.zeros(mlp_nparams(prm.hidden))
    dg0 = np.empty_like(g0) if want_dg0 else None
    L = lib().ora_unroll_grad(*_shape(g0), _p(g0), int(nsteps), C.byref(prm), _theta(theta),
                              _p(utx), _p(uty), _p(dth), _p(dg0))
    return L, dth, dg0


def mlp_collide_vjp(f, pb, prm, theta, Fx=0.0, Fy=0.0):
    """Single-node reverse mode of the learned collision: (dL/df_pre, dL/dtheta)."""
    f, pb = _f64(f), _f64(pb)
    fb = np.zeros(9)
    dth = np.zeros(mlp_nparams(prm.hidden))
    lib().ora_mlp_collide_vjp(_p(f), _p(pb), C.byref(prm), _theta(theta), float(Fx), float(Fy),
                              _p(fb), _p(dth))
    return fb, dth


def equilibrium_field(rho, ux, uy):
    """f = feq(rho, u) at every node, as a (B, 9, ny, nx) array."""
    rho, ux, uy = (_f64(a) for a in (rho, ux, uy))
    B, ny, nx = rho.shape
    out = np.empty((B, 9, ny, nx))
    lib().ora_feq_field(B, ny, nx, _p(rho), _p(ux), _p(uy), _p(out))
    return out


def structure_functions(ux, uy, rmax):
    """Longitudinal S^p(r), p = 1..6, r = 1..rmax, averaged over nodes and the two
    lattice directions (structure-function definition, SI section 3).
    Returns an array [6, rmax]; row p-1 is S^p."""
    ux, uy = _f64(ux), _f64(uy)
    B, ny, nx = ux.shape
    out = np.zeros(6 * rmax)
    lib().ora_structure_functions(B, ny, nx, _p(ux), _p(uy), int(rmax), _p(out))
    return out.reshape(6, rmax)


def energy_spectrum(ux, uy, kmax):
    """Shell-averaged kinetic energy spectrum of periodic fields [B, ny, nx]:
    E(k) = 1/2 sum over wavevectors with round(|k|) = k of |u_hat(k)|^2 / N^2,
    N = nx ny, averaged over the batch (so sum_k E(k) = <|u|^2>/2 when kmax
    covers every shell).  k in grid units: k_x in [-nx/2, nx/2), same in y.
    The FFT is numpy's (a library step); the binning is written out here."""
    ux, uy = _f64(ux), _f64(uy)
    B, ny, nx = ux.shape
    N = nx * ny
    E = np.zeros(kmax + 1)
    ky = np.fft.fftfreq(ny) * ny
    kx = np.fft.fftfreq(nx) * nx
    KY, KX = np.meshgrid(ky, kx, indexing="ij")
    shell = np.rint(np.sqrt(KX ** 2 + KY ** 2)).astype(int)
    for b in range(B):
        e = 0.5 * (np.abs(np.fft.fft2(ux[b])) ** 2 + np.abs(np.fft.fft2(uy[b])) ** 2) / N ** 2
        for s_, v in zip(shell.ravel(), e.ravel()):
            if s_ <= kmax:
                E[s_] += v
    return E / B


def _idx(idx):
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    return idx, idx.ctypes.data_as(C.POINTER(C.c_int))


def velocity_loss_subset(fpre, idx, utx, uty):
    """Velocity loss on the nodes idx (flat b*ny*nx + y*nx + x) and its gradient
    (Eq. S13 with the random subset of the unrolled training, velocity form)."""
    fpre, utx, uty = _f64(fpre), _f64(utx), _f64(uty)
    idx, pidx = _idx(idx)
    g = np.empty_like(fpre)
    L = lib().ora_velocity_loss_subset(*_shape(fpre), _p(fpre), pidx, len(idx), _p(utx), _p(uty),
                                       _p(g))
    return L, g


def population_loss_subset(g_post, idx, target):
    """Population loss of Eq. S13 on the nodes idx (sum over the subset and the
    nine populations, as printed) and its gradient w.r.t. g_post."""
    g_post, target = _f64(g_post), _f64(target)
    idx, pidx = _idx(idx)
    grad = np.empty_like(g_post)
    L = lib().ora_population_loss_subset(*_shape(g_post), _p(g_post), pidx, len(idx),
                                         _p(target), _p(grad))
    return L, grad


def subsample(f, cg):
    """Filter phi of SI section 2: every cg-th node along both axes."""
    f = _f64(f)
    B, ny, nx = _shape(f)
    out = np.empty((B, 9, ny // cg, nx // cg))
    lib().ora_subsample(B, ny, nx, int(cg), _p(f), _p(out))
    return out

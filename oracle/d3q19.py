"""FP64 CPU oracle of the paper's D3Q19 setting (``d3q19_oracle.c``).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle``: used by ``tests/``,
never by the library path.  Populations are float64 arrays (B, 19, nz, ny, nx);
the stored state of a run is the post-collision field g, and the pre-collision
populations of the next step are ``stream_pull(g)``.  Stencil and weights are
the paper's D3Q19 table, in its index order.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import lib as _lib_d2

BGK, SMAG, MLP = 0, 1, 2
WIDTHS = (300, 300, 100)
LEAKY_SLOPE = 0.01


class Params(C.Structure):
    _fields_ = [
        ("tau", C.c_double),
        ("smag_cs", C.c_double),
        ("smag_delta", C.c_double),
        ("force_amp", C.c_double),
        ("force_mode", C.c_int),
        ("h1", C.c_int),
        ("h2", C.c_int),
        ("h3", C.c_int),
        ("leaky_slope", C.c_double),
    ]


def params(tau, smag_cs=0.0, smag_delta=1.0, force_amp=0.0, force_mode=1, widths=WIDTHS,
           leaky_slope=LEAKY_SLOPE):
    h1, h2, h3 = widths
    return Params(float(tau), float(smag_cs), float(smag_delta), float(force_amp),
                  int(force_mode), int(h1), int(h2), int(h3), float(leaky_slope))


_sig_done = False


def lib():
    global _sig_done
    L = _lib_d2()
    if not _sig_done:
        d, i, pd, pi = C.c_double, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int)
        pp = C.POINTER(Params)
        sig = {
            "o3_lattice": (None, [pi, pi, pi, pd]),
            "o3_feq": (None, [d, d, d, d, pd]),
            "o3_stream_pull": (None, [i, i, i, i, pd, pd]),
            "o3_stream_push": (None, [i, i, i, i, pd, pd]),
            "o3_moments": (None, [i, i, i, i, pd, pd, pd]),
            "o3_force": (None, [pp, i, i, i, i, i, i, pd]),
            "o3_edm_force": (None, [d, pd, pd, pd]),
            "o3_smag_tau_eff": (d, [pd, d, d, d]),
            "o3_project": (None, [pd, pd]),
            "o3_mlp_nparams": (i, [i, i, i]),
            "o3_mlp_forward": (None, [pd, pp, pd, pd]),
            "o3_collide_node": (None, [i, pd, pd, pp, pd, pd]),
            "o3_collide": (None, [i, i, i, i, i, pd, pd, pp, pd]),
            "o3_step": (None, [i, i, i, i, i, pd, pd, pp, pd]),
            "o3_run": (None, [i, i, i, i, i, pd, i, pp, pd]),
            "o3_feq_field": (None, [i, i, i, i, pd, pd, pd]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _sig_done = True
    return L


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _shape(f):
    B, q, nz, ny, nx = f.shape
    assert q == 19
    return B, nz, ny, nx


def lattice():
    """(cx, cy, cz, w) of the paper's D3Q19 table."""
    cx, cy, cz = (C.c_int * 19)(), (C.c_int * 19)(), (C.c_int * 19)()
    w = np.empty(19)
    lib().o3_lattice(cx, cy, cz, _p(w))
    return np.array(cx), np.array(cy), np.array(cz), w


def feq(rho, u):
    out = np.empty(19)
    lib().o3_feq(float(rho), float(u[0]), float(u[1]), float(u[2]), _p(out))
    return out


def stream_pull(g):
    g = _f64(g)
    out = np.empty_like(g)
    lib().o3_stream_pull(*_shape(g), _p(g), _p(out))
    return out


def stream_push(f):
    f = _f64(f)
    out = np.empty_like(f)
    lib().o3_stream_push(*_shape(f), _p(f), _p(out))
    return out


def moments(f):
    """rho [B, nz, ny, nx] and u [B, 3, nz, ny, nx] (u = j / rho)."""
    f = _f64(f)
    B, nz, ny, nx = _shape(f)
    rho = np.empty((B, nz, ny, nx))
    u = np.empty((B, 3, nz, ny, nx))
    lib().o3_moments(B, nz, ny, nx, _p(f), _p(rho), _p(u))
    return rho, u


def force(prm, z, y, x, nz, ny, nx):
    out = np.empty(3)
    lib().o3_force(C.byref(prm), z, y, x, nz, ny, nx, _p(out))
    return out


def edm_force(rho, u, F):
    out = np.empty(19)
    lib().o3_edm_force(float(rho), _p(_f64(u)), _p(_f64(F)), _p(out))
    return out


def smag_tau_eff(f, tau0, cs, delta=1.0):
    return lib().o3_smag_tau_eff(_p(_f64(f)), tau0, cs, delta)


def project(o):
    o = _f64(o)
    out = np.empty(19)
    lib().o3_project(_p(o), _p(out))
    return out


def mlp_nparams(widths=WIDTHS):
    return lib().o3_mlp_nparams(*widths)


def mlp_forward(theta, x, prm):
    out = np.empty(19)
    lib().o3_mlp_forward(_p(_f64(theta)), C.byref(prm), _p(_f64(x)), _p(out))
    return out


def collide_node(kind, f, prm, theta=None, F=(0.0, 0.0, 0.0)):
    out = np.empty(19)
    th = _p(_f64(theta)) if theta is not None else None
    lib().o3_collide_node(kind, _p(_f64(f)), _p(out), C.byref(prm), th, _p(_f64(F)))
    return out


def collide(kind, fpre, prm, theta=None):
    fpre = _f64(fpre)
    out = np.empty_like(fpre)
    th = _p(_f64(theta)) if theta is not None else None
    lib().o3_collide(*_shape(fpre), kind, _p(fpre), _p(out), C.byref(prm), th)
    return out


def step(kind, g, prm, theta=None):
    g = _f64(g)
    out = np.empty_like(g)
    th = _p(_f64(theta)) if theta is not None else None
    lib().o3_step(*_shape(g), kind, _p(g), _p(out), C.byref(prm), th)
    return out


def run(kind, g, nsteps, prm, theta=None):
    g = _f64(g).copy()
    th = _p(_f64(theta)) if theta is not None else None
    lib().o3_run(*_shape(g), kind, _p(g), int(nsteps), C.byref(prm), th)
    return g


def equilibrium_field(rho, u):
    """rho [B, nz, ny, nx], u [B, 3, nz, ny, nx] -> feq populations."""
    rho, u = _f64(rho), _f64(u)
    B, nz, ny, nx = rho.shape
    out = np.empty((B, 19, nz, ny, nx))
    lib().o3_feq_field(B, nz, ny, nx, _p(rho), _p(u), _p(out))
    return out

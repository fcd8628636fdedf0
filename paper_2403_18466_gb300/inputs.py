"""Seeded synthetic inputs shared by the CUDA path and the oracle tests.

This module holds none of the lattice-Boltzmann arithmetic: it only makes
velocity fields, random numbers and network weights.  Both sides turn its
output into populations with their own equilibrium code.

Recipes (the paper's 3D HIT DNS data is not available; these stand in for it
with the structure the paper describes: a divergence-free turbulent field of
a few percent of the lattice speed, driven by a large-scale sine force):

* ``taylor_green``: u_x = -u0 cos(kx) sin(ky), u_y = u0 sin(kx) cos(ky).
* ``shear_wave``: u_x = u0 sin(k y), u_y = 0.
* ``random_velocity_field``: a random-phase, divergence-free 2D field built
  from a stream function with energy spectrum E(k) ~ k^4 exp(-2 (k/k0)^2),
  zero mean, scaled so that sqrt(<u_x^2 + u_y^2>/2) equals ``urms``.
* ``xavier_mlp``: Glorot-uniform weights (Glorot & Bengio 2010) for the
  9 -> h -> h -> 9 network, packed as W1[h][9], b1[h], W2[h][h], b2[h],
  W3[9][h], b3[9]; biases zero unless ``bias_scale`` is given.
"""
from __future__ import annotations

import os

import numpy as np

HIDDEN = 64


def taylor_green(n: int, u0: float, k: float):
    """Taylor-Green vortex on an n x n periodic grid; returns (rho, ux, uy)."""
    y, x = np.meshgrid(np.arange(n, dtype=np.float64), np.arange(n, dtype=np.float64),
                       indexing="ij")
    ux = -u0 * np.cos(k * x) * np.sin(k * y)
    uy = u0 * np.sin(k * x) * np.cos(k * y)
    return np.ones((n, n)), ux, uy


def shear_wave(n: int, u0: float, k: float):
    """u_x = u0 sin(k y) on an n x n periodic grid; returns (rho, ux, uy)."""
    y = np.arange(n, dtype=np.float64)[:, None] * np.ones((1, n))
    return np.ones((n, n)), u0 * np.sin(k * y), np.zeros((n, n))


def random_velocity_field(ny: int, nx: int, seed: int, k0: float = 8.0, urms: float = 0.02):
    """Random-phase divergence-free field; returns (rho, ux, uy) in float64.

    psi_hat(k) = A(|k|) exp(i theta_k) with |u_hat| ~ sqrt(E(k) / (pi k)),
    u_hat = i (k_y, -k_x) psi_hat; the real part of the inverse FFT is
    divergence-free to rounding.  Seeded numpy PCG64.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    ky = np.fft.fftfreq(ny) * ny
    kx = np.fft.fftfreq(nx) * nx
    KY, KX = np.meshgrid(ky, kx, indexing="ij")
    kk = np.sqrt(KX ** 2 + KY ** 2)
    E = kk ** 4 * np.exp(-2.0 * (kk / k0) ** 2)
    with np.errstate(divide="ignore", invalid="ignore"):
        amp_u = np.where(kk > 0, np.sqrt(E / (np.pi * np.maximum(kk, 1e-30))), 0.0)
        amp_psi = np.where(kk > 0, amp_u / np.maximum(kk, 1e-30), 0.0)
    theta = rng.uniform(0.0, 2.0 * np.pi, size=kk.shape)
    psi_hat = amp_psi * np.exp(1j * theta)
    # Nyquist rows/columns have no Hermitian partner: drop them so that the
    # real part stays divergence-free
    if ny % 2 == 0:
        psi_hat[ny // 2, :] = 0.0
    if nx % 2 == 0:
        psi_hat[:, nx // 2] = 0.0
    # scale wavenumbers to radians per lattice unit for the derivative
    sy, sx = 2.0 * np.pi / ny, 2.0 * np.pi / nx
    ux = np.real(np.fft.ifft2(1j * (KY * sy) * psi_hat))
    uy = np.real(np.fft.ifft2(-1j * (KX * sx) * psi_hat))
    ux -= ux.mean()
    uy -= uy.mean()
    rms = np.sqrt(0.5 * np.mean(ux ** 2 + uy ** 2))
    if rms > 0:
        ux *= urms / rms
        uy *= urms / rms
    return np.ones((ny, nx)), ux, uy


def random_velocity_field_3d(nz: int, ny: int, nx: int, seed: int, k0: float = 4.0,
                             urms: float = 0.02):
    """Seeded divergence-free 3D field: Gaussian random Fourier amplitudes with
    |u_hat| shaped by sqrt(E(k) / (4 pi k^2)), E(k) ~ k^4 exp(-2 (k/k0)^2), made
    solenoidal by removing the component along k, real part of the inverse FFT
    (Nyquist planes dropped), zero mean, scaled so that
    sqrt(<|u|^2> / 3) = urms.  Returns rho (ones), u [3, nz, ny, nx]."""
    rng = np.random.default_rng(seed)
    kz = np.fft.fftfreq(nz, 1.0 / nz)[:, None, None]
    ky = np.fft.fftfreq(ny, 1.0 / ny)[None, :, None]
    kx = np.fft.fftfreq(nx, 1.0 / nx)[None, None, :]
    k2 = kx ** 2 + ky ** 2 + kz ** 2
    k = np.sqrt(k2)
    spec = k ** 4 * np.exp(-2.0 * (k / k0) ** 2)
    amp = np.where(k > 0, np.sqrt(spec / (4 * np.pi * np.maximum(k2, 1))), 0.0)
    w = (rng.standard_normal((3, nz, ny, nx)) + 1j * rng.standard_normal((3, nz, ny, nx))) * amp
    kv = [np.broadcast_to(a, (nz, ny, nx)) for a in (kx, ky, kz)]
    kdotw = sum(kv[a] * w[a] for a in range(3))
    uh = np.stack([w[a] - kv[a] * kdotw / np.maximum(k2, 1) for a in range(3)])
    for n, kk in ((nx, kv[0]), (ny, kv[1]), (nz, kv[2])):
        if n % 2 == 0:
            uh[:, np.abs(kk) == n // 2] = 0.0
    u = np.real(np.fft.ifftn(uh, axes=(1, 2, 3)))
    u -= u.mean(axis=(1, 2, 3), keepdims=True)
    norm = np.sqrt(np.mean(np.sum(u ** 2, axis=0)) / 3.0)
    if norm == 0.0:
        raise ValueError("grid too small for a non-trivial solenoidal field")
    u *= urms / norm
    return np.ones((nz, ny, nx)), u


def xavier_mlp_widths(seed: int, widths, bias_scale: float = 0.0, gain: float = 1.0,
                      out_scale: float = 1.0):
    """Seeded Xavier-uniform weights of a 19 -> widths... -> 19 MLP, packed as
    W1[h1][19], b1, W2[h2][h1], b2, ..., W_out[19][h_last], b_out (float64)."""
    rng = np.random.default_rng(seed)
    dims = [19, *widths, 19]
    parts = []
    for layer, (nin, nout) in enumerate(zip(dims[:-1], dims[1:])):
        lim = gain * np.sqrt(6.0 / (nin + nout))
        Wl = rng.uniform(-lim, lim, (nout, nin))
        bl = rng.uniform(-bias_scale, bias_scale, nout) if bias_scale else np.zeros(nout)
        if layer == len(dims) - 2:
            Wl, bl = Wl / gain * out_scale, bl * out_scale
        parts += [Wl.ravel(), bl]
    return np.concatenate(parts)


def mlp_nparams(h: int = HIDDEN) -> int:
    return h * 9 + h + h * h + h + 9 * h + 9


def xavier_mlp(seed: int, h: int = HIDDEN, bias_scale: float = 0.0, gain: float = 1.0,
               out_scale: float = 1.0):
    """Packed float64 weights of the 9 -> h -> h -> 9 network (Glorot uniform).

    ``gain`` scales the two hidden layers' bounds, ``out_scale`` multiplies the
    output layer (W3 and b3), so that a strongly non-linear network can still
    produce a correction of the size of the non-equilibrium populations."""
    rng = np.random.Generator(np.random.PCG64(seed))

    def glorot(fan_out, fan_in):
        a = gain * np.sqrt(6.0 / (fan_in + fan_out))
        return rng.uniform(-a, a, size=(fan_out, fan_in))

    W1 = glorot(h, 9)
    W2 = glorot(h, h)
    W3 = glorot(9, h) / gain * out_scale
    b1, b2, b3 = (bias_scale * rng.uniform(-1.0, 1.0, size=m) for m in (h, h, 9))
    b3 = b3 * out_scale
    return np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3.ravel(), b3])


def unpack_mlp(theta, h: int = HIDDEN):
    """Split a packed parameter vector into (W1, b1, W2, b2, W3, b3) views."""
    theta = np.asarray(theta)
    sizes = [h * 9, h, h * h, h, 9 * h, 9]
    shapes = [(h, 9), (h,), (h, h), (h,), (9, h), (9,)]
    out, o = [], 0
    for s, shp in zip(sizes, shapes):
        out.append(theta[o:o + s].reshape(shp))
        o += s
    return tuple(out)


def noise(shape, seed: int, scale: float):
    """Uniform noise in [-scale, scale] (float64), seeded."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return scale * rng.uniform(-1.0, 1.0, size=shape)


def save_weights(theta, path):
    """Write a packed weight vector (torch tensor or array) as float32 .npy."""
    a = theta.detach().cpu().numpy() if hasattr(theta, "detach") else np.asarray(theta)
    np.save(path, a.astype(np.float32))


def load_weights(path, device=None):
    """Read a packed weight vector written by save_weights; a CUDA float32
    tensor if `device` is given, else a float64 numpy array."""
    a = np.load(path).astype(np.float64)
    if device is None:
        return a
    import torch
    return torch.tensor(a, dtype=torch.float32, device=device)


TRAINED_WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights",
                               "d2q9_les_cg8.npy")


def trained_mlp(device=None):
    """Weights of the 9 -> 64 -> 64 -> 9 collision network trained by this
    library (``python -m paper_2403_18466_gb300.train --precision f32 --lr 1e-4
    --epochs 400 --save ...``: 2048^2 BGK DNS, tau 0.503, box filter x8 to 256^2
    LES at tau' = 0.500375, 32 trajectories unrolled 16 steps, checkpoint every
    4, velocity loss 7.18e-8 -> 3.90e-8 against 7.26e-8 for plain BGK LES).
    Same packing as xavier_mlp; float64 numpy, or a CUDA float32 tensor."""
    return load_weights(TRAINED_WEIGHTS, device)

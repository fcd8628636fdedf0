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

"""Pins of the oracle's flow diagnostics (SI section 3 and the energy spectra of
the main text): closed forms for a single Fourier mode and Parseval's identity."""
import numpy as np

import oracle
from paper_2403_18466_gb300 import inputs


def _mode(n, A, k0):
    x = np.arange(n)[None, :] * np.ones((n, 1))
    return A * np.sin(2 * np.pi * k0 * x / n)[None], np.zeros((1, n, n))


def test_structure_functions_single_mode_closed_forms():
    n, A, k0, rmax = 32, 0.03, 3, 10
    ux, uy = _mode(n, A, k0)
    S = oracle.structure_functions(ux, uy, rmax)
    r = np.arange(1, rmax + 1)
    s = np.sin(np.pi * k0 * r / n)  # sin(kappa r / 2)
    # du = 2 A cos(kappa (x + r/2)) sin(kappa r / 2) along x, 0 along y (halved by the average)
    assert np.allclose(S[0], 0.0, atol=1e-17)
    assert np.allclose(S[1], 0.5 * 2 * A ** 2 * s ** 2, rtol=1e-12)
    assert np.allclose(S[2], 0.0, atol=1e-18)
    assert np.allclose(S[3], 0.5 * 6 * A ** 4 * s ** 4, rtol=1e-12)
    assert np.allclose(S[5], 0.5 * 20 * A ** 6 * s ** 6, rtol=1e-12)


def test_structure_functions_match_direct_numpy_average():
    rho, ux, uy = inputs.random_velocity_field(24, 20, seed=5, k0=3.0)
    S = oracle.structure_functions(ux[None], uy[None], 7)
    for r in (1, 4, 7):
        dx = np.roll(ux, -r, axis=1) - ux
        dy = np.roll(uy, -r, axis=0) - uy
        for p in range(1, 7):
            scale = np.mean(np.abs(dx) ** p + np.abs(dy) ** p)
            assert abs(S[p - 1, r - 1] - 0.5 * (np.mean(dx ** p) + np.mean(dy ** p))) <= 1e-12 * scale


def test_energy_spectrum_single_mode_and_parseval():
    n, A, k0 = 32, 0.05, 4
    ux, uy = _mode(n, A, k0)
    E = oracle.energy_spectrum(ux, uy, n)
    assert np.isclose(E[k0], A ** 2 / 4, rtol=1e-12)
    assert np.allclose(np.delete(E, k0), 0.0, atol=1e-20)
    rho, vx, vy = inputs.random_velocity_field(32, 32, seed=2, k0=5.0, urms=0.02)
    E = oracle.energy_spectrum(vx[None], vy[None], 32)  # covers every shell up to 16 sqrt 2
    assert np.isclose(E.sum(), 0.5 * np.mean(vx ** 2 + vy ** 2), rtol=1e-12)

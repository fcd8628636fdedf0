"""Pins of the oracle's full time stepping against flows with known solutions.

* Taylor-Green vortex: amplitude decays as exp(-2 nu k^2 t), nu = cs^2 (tau - 1/2)
  (Eq. S6), fitted over t in [100, 1000] on 64^2 at tau = 0.6 (the 64^2
  Taylor-Green configuration).
* Shear wave: amplitude decays as exp(-nu k^2 t).
* Kolmogorov flow: under the forcing F_x = F0 sin(k y) the steady laminar
  solution is u_x = F0 sin(k y) / (nu k^2) (Stokes flow), with the EDM
  velocity (j + F/2)/rho.
* Global mass is conserved and each collision adds F(y) per node of row y.
* Smagorinsky with C_s = 0 reproduces BGK over a whole run.
"""
import numpy as np

import oracle
from paper_2403_18466_gb300 import inputs

CX, CY, W = oracle.lattice()


def _g_from_u(rho, ux, uy):
    """Post-collision state whose streamed (pre-collision) populations are feq."""
    f = oracle.equilibrium_field(rho[None], ux[None], uy[None])
    return oracle.stream_push(f)


def _fit_rate(ts, amps):
    return -np.polyfit(ts, np.log(amps), 1)[0]


def test_taylor_green_decay_rate():
    n, tau, u0 = 64, 0.6, 0.01
    k = 2 * np.pi / n
    rho, ux, uy = inputs.taylor_green(n, u0, k)
    g = _g_from_u(rho, ux, uy)
    prm = oracle.params(tau)
    ts, amps = [], []
    mass0 = oracle.stream_pull(g).sum()
    for t in range(0, 1001, 100):
        if t > 0:
            g = oracle.run(oracle.BGK, g, 100, prm)
        if t >= 100:
            _, vx, vy = oracle.moments(oracle.stream_pull(g))
            # project on the initial mode shape
            amps.append(np.sum(vx[0] * ux) / np.sum(ux * ux) * u0)
            ts.append(t)
    nu_fit = _fit_rate(np.array(ts), np.array(amps)) / (2 * k * k)
    nu = oracle.viscosity(tau)
    assert abs(nu_fit / nu - 1) < 0.02
    # predicted ratio at t = 1000 from the closed form
    assert abs(amps[-1] / u0 - np.exp(-2 * nu * k * k * 1000)) < 0.02 * np.exp(-2 * nu * k * k * 1000)
    assert abs(oracle.stream_pull(g).sum() / mass0 - 1) < 1e-13


def test_shear_wave_decay_rate():
    n, tau, u0 = 32, 0.8, 1e-3
    k = 2 * np.pi / n
    rho, ux, uy = inputs.shear_wave(n, u0, k)
    g = _g_from_u(rho, ux, uy)
    prm = oracle.params(tau)
    ts, amps = [], []
    for t in range(0, 601, 50):
        if t > 0:
            g = oracle.run(oracle.BGK, g, 50, prm)
        if t >= 50:
            _, vx, _ = oracle.moments(oracle.stream_pull(g))
            amps.append(np.sum(vx[0] * ux) / np.sum(ux * ux) * u0)
            ts.append(t)
    nu_fit = _fit_rate(np.array(ts), np.array(amps)) / (k * k)
    assert abs(nu_fit / oracle.viscosity(tau) - 1) < 0.02


def test_kolmogorov_steady_state_and_momentum_budget():
    ny, nx, tau, F0, m = 32, 4, 0.6, 1e-6, 1
    k = 2 * np.pi * m / ny
    nu = oracle.viscosity(tau)
    rho = np.ones((ny, nx))
    z = np.zeros((ny, nx))
    g = _g_from_u(rho, z, z)
    prm = oracle.params(tau, force_amp=F0, force_mode=m)
    # momentum budget of one step, row by row: the collision adds F(y) at
    # every node of row y (before streaming moves it between rows)
    f0 = oracle.stream_pull(g)
    g1 = oracle.step(oracle.BGK, g, prm)
    y = np.arange(ny)
    Fy = F0 * np.sin(2 * np.pi * m * y / ny)
    jx0 = np.einsum("biyx,i->y", f0, CX)
    jx1 = np.einsum("biyx,i->y", g1, CX)
    assert np.allclose(jx1 - jx0, nx * Fy, rtol=0, atol=5e-16)  # row sums of O(0.1) terms
    # steady Stokes solution after ~10 viscous times 1/(nu k^2)
    g = oracle.run(oracle.BGK, g, int(12 / (nu * k * k)), prm)
    f = oracle.stream_pull(g)
    r, vx, vy = oracle.moments(f)
    vphys = vx[0] + Fy[:, None] / (2 * r[0])
    expect = F0 * np.sin(k * y) / (nu * k * k)
    err = np.abs(vphys - expect[:, None]).max() / np.abs(expect).max()
    assert err < 0.01
    assert np.abs(vy).max() < 1e-9 * np.abs(expect).max()  # rounding drift only


def test_smagorinsky_zero_constant_run_equals_bgk_run():
    rho, ux, uy = inputs.random_velocity_field(16, 16, seed=1, k0=3.0, urms=0.02)
    g = _g_from_u(rho, ux, uy)
    a = oracle.run(oracle.SMAG, g, 20, oracle.params(0.51, smag_cs=0.0, force_amp=1e-5, force_mode=1))
    b = oracle.run(oracle.BGK, g, 20, oracle.params(0.51, force_amp=1e-5, force_mode=1))
    assert np.array_equal(a, b)


def test_smagorinsky_dissipates_more_than_bgk():
    """A positive eddy viscosity can only remove kinetic energy faster."""
    rho, ux, uy = inputs.random_velocity_field(32, 32, seed=2, k0=6.0, urms=0.05)
    g = _g_from_u(rho, ux, uy)
    ke = []
    for kind, cs in ((oracle.BGK, 0.0), (oracle.SMAG, 0.2)):
        h = oracle.run(kind, g, 50, oracle.params(0.505, smag_cs=cs))
        _, vx, vy = oracle.moments(oracle.stream_pull(h))
        ke.append(np.sum(vx ** 2 + vy ** 2))
    assert ke[1] < ke[0]

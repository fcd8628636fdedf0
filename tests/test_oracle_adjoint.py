"""Pins of the oracle's hand-written reverse mode (unrolled training, SI sec. 2).

The adjoint is pinned by central finite differences of the oracle's own
forward map in FP64 (an independent check: differences of forward values
need none of the reverse-mode code), per node and over whole unrolled
trajectories, including the 32^2 gradient check.
"""
import numpy as np
import pytest

import oracle
from paper_2403_18466_gb300 import inputs

CX, CY, W = oracle.lattice()


def _node(seed):
    f = oracle.feq(1.05, 0.04, -0.03)
    return f * (1 + inputs.noise(9, seed, 0.3))


def test_node_vjp_by_central_differences():
    prm = oracle.params(0.57)
    theta = inputs.xavier_mlp(2, bias_scale=0.5, gain=5.0)
    f = _node(1)
    pb = inputs.noise(9, 2, 1.0)
    Fx, Fy = 2e-3, -1e-3
    fb, dth = oracle.mlp_collide_vjp(f, pb, prm, theta, Fx, Fy)

    def J(ff, th):
        return pb @ oracle.collide_node(oracle.MLP, ff, prm, th, Fx, Fy)

    eps = 1e-6
    for k in range(9):
        e = np.zeros(9)
        e[k] = eps
        fd = (J(f + e, theta) - J(f - e, theta)) / (2 * eps)
        assert abs(fd - fb[k]) < 1e-8 * (1 + abs(fb[k]))
    rng = np.random.default_rng(0)
    for k in list(rng.choice(theta.size, 30, replace=False)) + [0, 575, 640, 4735, 5375, 5384]:
        e = np.zeros_like(theta)
        e[k] = eps
        fd = (J(f, theta + e) - J(f, theta - e)) / (2 * eps)
        assert abs(fd - dth[k]) < 1e-8 * (1 + abs(dth[k]))


def _trajectory_case(n, B, seed):
    g = []
    for b in range(B):
        rho, ux, uy = inputs.random_velocity_field(n, n, seed=seed + b, k0=2.0, urms=0.04)
        f = oracle.equilibrium_field(rho[None], ux[None], uy[None])
        g.append(oracle.stream_push(f * (1 + inputs.noise(f.shape, seed + 10 + b, 0.05))))
    g = np.concatenate(g, 0)
    utx = inputs.noise((B, n, n), seed + 20, 0.05)
    uty = inputs.noise((B, n, n), seed + 21, 0.05)
    return g, utx, uty


@pytest.mark.parametrize("n,B,steps", [(6, 2, 3), (32, 1, 2)])
def test_unrolled_gradient_by_central_differences(n, B, steps):
    prm = oracle.params(0.6, force_amp=1e-4, force_mode=1)
    theta = inputs.xavier_mlp(3, bias_scale=0.3, gain=4.0)
    g, utx, uty = _trajectory_case(n, B, 40)
    L, dth, dg0 = oracle.unroll_grad(g, steps, prm, theta, utx, uty)
    assert np.isclose(L, oracle.unroll_loss(g, steps, prm, theta, utx, uty), rtol=1e-14)
    rng = np.random.default_rng(1)

    def central(fun, eps):
        # Richardson-extrapolated central difference, error O(eps^4)
        d1 = (fun(eps) - fun(-eps)) / (2 * eps)
        d2 = (fun(eps / 2) - fun(-eps / 2)) / eps
        return (4 * d2 - d1) / 3

    for trial in range(3 if n <= 8 else 2):
        d = rng.normal(size=theta.size)
        d /= np.linalg.norm(d)
        fd = central(lambda h: oracle.unroll_loss(g, steps, prm, theta + h * d, utx, uty), 1e-4)
        assert abs(fd - dth @ d) <= 1e-6 * np.linalg.norm(dth)
        e = rng.normal(size=g.shape)
        e /= np.linalg.norm(e)
        fd = central(lambda h: oracle.unroll_loss(g + h * e, steps, prm, theta, utx, uty), 1e-5)
        assert abs(fd - np.sum(dg0 * e)) <= 1e-6 * np.linalg.norm(dg0)


def test_adjoint_dot_product_identity_of_streaming():
    """<S a, b> = <a, S^T b> with S^T the push: the transpose used by the adjoint."""
    a = inputs.noise((2, 9, 5, 7), 1, 1.0)
    b = inputs.noise((2, 9, 5, 7), 2, 1.0)
    assert np.isclose(np.sum(oracle.stream_pull(a) * b), np.sum(a * oracle.stream_push(b)),
                      rtol=1e-14)

"""Pins of the oracle's collision operators (BGK, Smagorinsky, EDM forcing,
projection and the learned collision).

What fixes each one independently of the oracle's code:
  * conservation of mass and momentum (Eqs. S11-S12 and the LBM moments);
  * the equilibrium as a fixed point of collision;
  * the Chapman-Enskog relation Pi^neq = -2 rho cs^2 tau S, which turns a
    prescribed strain into a state whose Smagorinsky viscosity is known;
  * homogeneity of degree one of every collision in f (intensive input
    (f - feq)/rho, extensive correction rho * ohat);
  * special cases that reduce to BGK (C_s = 0, F = 0, W3 = b3 = 0, an output
    inside span{1, c_x, c_y});
  * a numpy restatement of the 9 -> 64 -> 64 -> 9 network.
"""
import numpy as np
import pytest

import oracle
from paper_2403_18466_gb300 import inputs

CS2 = 1.0 / 3.0
CX, CY, W = oracle.lattice()
C2 = np.stack([CX, CY], 1).astype(float)


def _node(seed, rho=1.0, u=(0.03, -0.02), neq=0.01):
    f = oracle.feq(rho, *u)
    return f + inputs.noise(9, seed, neq) * W * 9


def _mass_mom(f):
    return f.sum(), f @ C2


@pytest.mark.parametrize("kind", [oracle.BGK, oracle.SMAG, oracle.MLP])
def test_collision_conserves_mass_and_momentum(kind):
    prm = oracle.params(0.6, smag_cs=0.1)
    theta = inputs.xavier_mlp(3, bias_scale=0.5, gain=3.0)
    for s in range(5):
        f = _node(s, rho=0.9 + 0.05 * s)
        q = oracle.collide_node(kind, f, prm, theta)
        m0, j0 = _mass_mom(f)
        m1, j1 = _mass_mom(q)
        # FP64 rounding of a sum of 9 terms of size max|q - f| (+ |f|)
        tol = 16 * np.finfo(float).eps * (np.abs(q - f).max() + np.abs(f).max())
        assert abs(m1 - m0) <= tol
        assert np.allclose(j1, j0, rtol=0, atol=tol)


@pytest.mark.parametrize("kind", [oracle.BGK, oracle.SMAG, oracle.MLP])
def test_equilibrium_is_fixed_point(kind):
    prm = oracle.params(0.55, smag_cs=0.17)
    theta = inputs.xavier_mlp(5, bias_scale=0.0)  # zero biases: MLP(0) = 0
    for rho, u in [(1.0, (0.0, 0.0)), (1.2, (0.04, 0.07)), (0.8, (-0.1, 0.02))]:
        f = oracle.feq(rho, *u)
        assert np.allclose(oracle.collide_node(kind, f, prm, theta), f, rtol=0, atol=2e-15)


@pytest.mark.parametrize("kind", [oracle.BGK, oracle.SMAG, oracle.MLP])
def test_collision_is_homogeneous_degree_one(kind):
    prm = oracle.params(0.6, smag_cs=0.2)
    theta = inputs.xavier_mlp(7, bias_scale=0.3, gain=4.0)
    f = _node(11, neq=0.05)
    q = oracle.collide_node(kind, f, prm, theta)
    for lam in (0.5, 2.0, 3.7):
        assert np.allclose(oracle.collide_node(kind, lam * f, prm, theta), lam * q, rtol=1e-13,
                           atol=0)


def test_bgk_relaxes_nonequilibrium_by_one_minus_one_over_tau():
    """Eq. S3: f_post - feq = (1 - 1/tau)(f - feq), with feq of the unchanged moments."""
    for tau in (0.51, 0.6, 1.0, 1.7):
        prm = oracle.params(tau)
        f = _node(2, rho=1.1, neq=0.03)
        rho = f.sum()
        u = f @ C2 / rho
        fe = oracle.feq(rho, *u)
        q = oracle.collide_node(oracle.BGK, f, prm)
        assert np.allclose(q - fe, (1 - 1 / tau) * (f - fe), rtol=0, atol=1e-15)
    # tau = 1 lands exactly on the equilibrium
    q = oracle.collide_node(oracle.BGK, _node(3), oracle.params(1.0))
    f = _node(3)
    assert np.allclose(q, oracle.feq(f.sum(), *(f @ C2 / f.sum())), atol=1e-15)


def test_edm_force_momentum_and_mass():
    """Eq. S5: the EDM term adds exactly F to the momentum and no mass."""
    for rho, ux, uy, Fx, Fy in [(1.0, 0.01, 0.0, 1e-5, 0.0), (0.9, -0.05, 0.03, 2e-3, -1e-3)]:
        fe = oracle.edm_force(rho, ux, uy, Fx, Fy)
        assert abs(fe.sum()) < 1e-16
        assert np.allclose(fe @ C2, [Fx, Fy], rtol=0, atol=1e-16)  # cancellation of O(0.1) terms
    assert np.array_equal(oracle.edm_force(1.0, 0.1, 0.1, 0.0, 0.0), np.zeros(9))


@pytest.mark.parametrize("kind", [oracle.BGK, oracle.SMAG, oracle.MLP])
def test_forced_collision_adds_exactly_F(kind):
    prm = oracle.params(0.6, smag_cs=0.1)
    theta = inputs.xavier_mlp(9, bias_scale=0.2, gain=2.0)
    f = _node(4, neq=0.02)
    Fx, Fy = 3e-4, -2e-4
    q = oracle.collide_node(kind, f, prm, theta, Fx, Fy)
    q0 = oracle.collide_node(kind, f, prm, theta)
    assert abs(q.sum() - f.sum()) < 1e-15
    assert np.allclose(q @ C2 - f @ C2, [Fx, Fy], rtol=1e-11, atol=1e-17)
    # forcing is the EDM term added after the collision
    rho = f.sum()
    u = f @ C2 / rho
    assert np.allclose(q - q0, oracle.edm_force(rho, *u, Fx, Fy), rtol=0, atol=1e-15)


def test_smagorinsky_with_zero_constant_is_bgk():
    f = _node(5, neq=0.04)
    a = oracle.collide_node(oracle.SMAG, f, oracle.params(0.51, smag_cs=0.0))
    b = oracle.collide_node(oracle.BGK, f, oracle.params(0.51))
    assert np.array_equal(a, b)


@pytest.mark.parametrize("rho,Cs,delta", [(1.0, 0.1, 1.0), (1.3, 0.2, 1.0), (0.8, 0.15, 2.0)])
def test_smagorinsky_viscosity_from_chapman_enskog_state(rho, Cs, delta):
    """Build the Chapman-Enskog state of a prescribed strain S relaxed with
    tau*: f = feq + f1, f1_i = -(w_i rho tau*/cs^2)(c_i c_i - cs^2 I):S, so that
    Pi^neq = -2 rho cs^2 tau* S.  The Smagorinsky model must then return
    tau_eff = tau* when tau0 is chosen so that nu_eff = nu0 + (Cs Delta)^2 |S|
    (Eq. S7 with |S| = sqrt(2 S:S))."""
    S = np.array([[2e-4, -3e-4], [-3e-4, -1e-4]])
    u = np.array([0.02, -0.01])
    tau_star = 0.58
    absS = np.sqrt(2.0 * np.sum(S * S))
    nu_star = CS2 * (tau_star - 0.5)
    nu0 = nu_star - (Cs * delta) ** 2 * absS
    tau0 = nu0 / CS2 + 0.5
    Q = np.einsum("ia,ib->iab", C2, C2) - CS2 * np.eye(2)[None]
    f1 = -(W * rho * tau_star / CS2) * np.einsum("iab,ab->i", Q, S)
    f = oracle.feq(rho, *u) + f1
    Pi = np.einsum("i,ia,ib->ab", f1, C2, C2)
    assert np.allclose(Pi, -2 * rho * CS2 * tau_star * S, rtol=1e-13, atol=0)
    t = oracle.smag_tau_eff(f, tau0, Cs, delta)
    assert abs(t - tau_star) < 1e-13


def test_projection_is_orthogonal_projector_removing_conserved_span():
    rng = np.random.default_rng(0)
    one = np.ones(9)
    for v in (one, CX.astype(float), CY.astype(float)):
        assert np.allclose(oracle.project(v), 0.0, atol=1e-15)
    P = np.stack([oracle.project(e) for e in np.eye(9)], 1)
    assert np.allclose(P @ P, P, atol=1e-15)
    assert np.allclose(P, P.T, atol=1e-15)
    assert np.isclose(np.trace(P), 6.0, atol=1e-14)  # rank 9 - 3
    for _ in range(5):
        o = rng.normal(size=9)
        oh = oracle.project(o)
        assert abs(oh.sum()) < 1e-15 * 10 and np.allclose(oh @ C2, 0.0, atol=1e-15 * 10)
        # removes exactly a combination of 1, c_x, c_y
        r = o - oh
        coef, *_ = np.linalg.lstsq(np.stack([one, CX, CY], 1).astype(float), r, rcond=None)
        assert np.allclose(np.stack([one, CX, CY], 1) @ coef, r, atol=1e-15)


def _np_mlp(theta, x, h=64):
    """Independent numpy restatement of the 9 -> h -> h -> 9 tanh network."""
    W1, b1, W2, b2, W3, b3 = inputs.unpack_mlp(theta, h)
    return W3 @ np.tanh(W2 @ np.tanh(W1 @ x + b1) + b2) + b3


def test_mlp_forward_matches_numpy_restatement():
    for seed in range(3):
        theta = inputs.xavier_mlp(seed, bias_scale=0.4, gain=2.0)
        x = inputs.noise(9, 100 + seed, 0.5)
        assert np.allclose(oracle.mlp_forward(theta, x), _np_mlp(theta, x), rtol=1e-14,
                           atol=1e-15)
    # a tiny width exercises the general-h code path
    theta = inputs.xavier_mlp(9, h=5, bias_scale=0.1)
    x = inputs.noise(9, 7, 1.0)
    assert np.allclose(oracle.mlp_forward(theta, x, h=5), _np_mlp(theta, x, h=5), rtol=1e-14)


def test_learned_collision_with_zero_output_layer_is_bgk():
    theta = inputs.xavier_mlp(4, bias_scale=0.5, gain=2.0)
    W1, b1, W2, b2, W3, b3 = inputs.unpack_mlp(theta)
    W3[:] = 0.0
    b3[:] = 0.0
    prm = oracle.params(0.6)
    f = _node(8, neq=0.05)
    assert np.array_equal(oracle.collide_node(oracle.MLP, f, prm, theta),
                          oracle.collide_node(oracle.BGK, f, prm))


def test_learned_collision_output_in_conserved_span_is_bgk():
    theta = inputs.xavier_mlp(4, bias_scale=0.5, gain=2.0)
    W1, b1, W2, b2, W3, b3 = inputs.unpack_mlp(theta)
    W3[:] = 0.0
    b3[:] = 0.3 - 0.2 * CX + 0.7 * CY
    prm = oracle.params(0.6)
    f = _node(9, neq=0.05)
    assert np.allclose(oracle.collide_node(oracle.MLP, f, prm, theta),
                       oracle.collide_node(oracle.BGK, f, prm), rtol=0, atol=1e-15)


def test_learned_collision_constant_output_is_scaled_projected_correction():
    """With W3 = 0 the network output is the constant b3, so the learned
    collision (Eq. S10) reduces to BGK + (rho/tau) P b3: pins the rho/tau
    scale and the projection together."""
    theta = inputs.xavier_mlp(4)
    W1, b1, W2, b2, W3, b3 = inputs.unpack_mlp(theta)
    W3[:] = 0.0
    b3[:] = inputs.noise(9, 5, 1e-3)
    f = _node(10, rho=1.4, neq=0.02)
    for tau in (0.52, 0.8):
        prm = oracle.params(tau)
        d = oracle.collide_node(oracle.MLP, f, prm, theta) - oracle.collide_node(oracle.BGK, f, prm)
        # the span-free part of b3, computed by least squares (independent of ora_project)
        A = np.stack([np.ones(9), CX, CY], 1).astype(float)
        coef, *_ = np.linalg.lstsq(A, b3, rcond=None)
        assert np.allclose(d, (f.sum() / tau) * (b3 - A @ coef), rtol=1e-12, atol=1e-18)

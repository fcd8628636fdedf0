"""D8 lattice-symmetry pins of the oracle, and the box filter's and loss's pins.

* BGK and Smagorinsky steps commute with the 8 symmetries of the square
  lattice (rotations by 90 degrees and reflections), forcing off.  The learned
  collision is not built equivariant (the paper's network is a plain MLP), so
  only its equivariance defect is computed, never asserted.
* Box filter: returns a block-constant field unchanged, conserves mass,
  agrees with a numpy reshape-mean, and commutes with free streaming
  (cg fine steps move a population by one coarse cell).
* Velocity loss: zero at the target, gradient equal to central differences.
* Subset losses (velocity and population forms of Eq. S13 on a node subset):
  the all-node velocity subset loss equals the full-field loss, the values
  equal a numpy gather, gradients vanish off the subset and match central
  differences on it.  Subsampling filter: a strided numpy slice.
"""
import numpy as np
import pytest

import oracle
from paper_2403_18466_gb300 import inputs

CX, CY, W = oracle.lattice()

D8 = [np.array(m) for m in ([[1, 0], [0, 1]], [[0, -1], [1, 0]], [[-1, 0], [0, -1]],
                            [[0, 1], [-1, 0]], [[1, 0], [0, -1]], [[-1, 0], [0, 1]],
                            [[0, 1], [1, 0]], [[0, -1], [-1, 0]])]


def _transform(f, T):
    """(T f)_{pi(i)}(T x) = f_i(x) with c_{pi(i)} = T c_i, on an n x n periodic grid."""
    B, q, n, n2 = f.shape
    assert n == n2
    out = np.empty_like(f)
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    xn = (T[0, 0] * x + T[0, 1] * y) % n
    yn = (T[1, 0] * x + T[1, 1] * y) % n
    for i in range(9):
        c = T @ np.array([CX[i], CY[i]])
        j = [k for k in range(9) if CX[k] == c[0] and CY[k] == c[1]][0]
        out[:, j, yn, xn] = f[:, i, y, x]
    return out


def _state(n, seed):
    rho, ux, uy = inputs.random_velocity_field(n, n, seed=seed, k0=3.0, urms=0.05)
    f = oracle.equilibrium_field(rho[None], ux[None], uy[None])
    return f * (1 + inputs.noise(f.shape, seed + 1, 0.02))


@pytest.mark.parametrize("kind", [oracle.BGK, oracle.SMAG])
def test_step_is_d8_equivariant(kind):
    g = _state(12, 3)
    prm = oracle.params(0.52, smag_cs=0.3)
    ref = oracle.run(kind, g, 3, prm)
    for T in D8:
        a = oracle.run(kind, _transform(g, T), 3, prm)
        assert np.allclose(a, _transform(ref, T), rtol=0, atol=1e-14 * np.abs(ref).max())


def test_transform_is_a_group_action():
    """The test's own transform: composition and inverse (guards the pin above)."""
    g = _state(6, 5)
    R = D8[1]
    assert np.array_equal(_transform(_transform(_transform(_transform(g, R), R), R), R), g)
    M = D8[4]
    assert np.array_equal(_transform(_transform(g, M), M), g)
    assert not np.array_equal(_transform(g, R), g)


def test_learned_collision_equivariance_defect_is_finite():
    """Reported, not asserted: the plain MLP is not D8-equivariant."""
    g = _state(8, 7)
    prm = oracle.params(0.6)
    theta = inputs.xavier_mlp(1, bias_scale=0.1, gain=3.0)
    ref = oracle.step(oracle.MLP, g, prm, theta)
    d = max(np.abs(oracle.step(oracle.MLP, _transform(g, T), prm, theta) - _transform(ref, T)).max()
            for T in D8)
    assert np.isfinite(d)


def test_box_filter_pins():
    cg, B, NY, NX = 4, 2, 3, 5
    coarse = 0.1 + inputs.noise((B, 9, NY, NX), 1, 0.05)
    fine = np.repeat(np.repeat(coarse, cg, axis=2), cg, axis=3)
    assert np.allclose(oracle.box_filter(fine, cg), coarse, rtol=1e-15)
    f = 0.1 + inputs.noise((B, 9, NY * cg, NX * cg), 2, 0.05)
    c = oracle.box_filter(f, cg)
    assert np.isclose(c.sum() * cg * cg, f.sum(), rtol=1e-14)
    ref = f.reshape(B, 9, NY, cg, NX, cg).mean(axis=(3, 5))
    assert np.allclose(c, ref, rtol=1e-14)


def test_box_filter_commutes_with_free_streaming():
    cg = 8
    f = 0.1 + inputs.noise((1, 9, 4 * cg, 3 * cg), 3, 0.05)
    s = f
    for _ in range(cg):
        s = oracle.stream_pull(s)
    assert np.allclose(oracle.box_filter(s, cg), oracle.stream_pull(oracle.box_filter(f, cg)),
                       rtol=1e-14)


def test_velocity_loss_zero_at_target_and_gradient_by_central_differences():
    B, ny, nx = 2, 3, 4
    rho, ux, uy = (np.ones((B, ny, nx)), inputs.noise((B, ny, nx), 4, 0.05),
                   inputs.noise((B, ny, nx), 5, 0.05))
    f = oracle.equilibrium_field(rho, ux, uy) + inputs.noise((B, 9, ny, nx), 6, 0.01)
    _, vx, vy = oracle.moments(f)
    assert oracle.velocity_loss(f, vx, vy) == 0.0
    utx, uty = inputs.noise((B, ny, nx), 7, 0.05), inputs.noise((B, ny, nx), 8, 0.05)
    # closed form of the mean: 1/(2NB) sum |u - u_t|^2
    L = oracle.velocity_loss(f, utx, uty)
    assert np.isclose(L, 0.5 * np.mean((vx - utx) ** 2 + (vy - uty) ** 2), rtol=1e-14)
    G = oracle.velocity_loss_grad(f, utx, uty)
    eps = 1e-6
    for idx in [(0, 0, 0, 0), (1, 5, 2, 3), (0, 8, 1, 2), (1, 3, 0, 1)]:
        fp, fm = f.copy(), f.copy()
        fp[idx] += eps
        fm[idx] -= eps
        fd = (oracle.velocity_loss(fp, utx, uty) - oracle.velocity_loss(fm, utx, uty)) / (2 * eps)
        assert abs(fd - G[idx]) < 1e-7 * np.abs(G).max()


def test_subset_losses_definitions_and_gradients():
    B, ny, nx = 2, 6, 7
    rho, ux, uy = (np.ones((B, ny, nx)), inputs.noise((B, ny, nx), 14, 0.05),
                   inputs.noise((B, ny, nx), 15, 0.05))
    f = oracle.equilibrium_field(rho, ux, uy) + inputs.noise((B, 9, ny, nx), 16, 0.01)
    utx, uty = inputs.noise((B, ny, nx), 17, 0.05), inputs.noise((B, ny, nx), 18, 0.05)
    idx = np.array([0, 5, 17, 43, 60, 83])
    L, G = oracle.velocity_loss_subset(f, idx, utx, uty)
    # the full-field loss is the subset loss with every node (same normalisation)
    Lall, _ = oracle.velocity_loss_subset(f, np.arange(B * ny * nx), utx, uty)
    assert np.isclose(Lall, oracle.velocity_loss(f, utx, uty), rtol=1e-14)
    _, vx, vy = oracle.moments(f)
    flat = lambda a: a.reshape(-1)
    ref = 0.5 * np.mean((flat(vx)[idx] - flat(utx)[idx]) ** 2 + (flat(vy)[idx] - flat(uty)[idx]) ** 2)
    assert np.isclose(L, ref, rtol=1e-14)
    # gradient is zero off the subset and matches central differences on it
    mask = np.zeros(B * ny * nx, bool)
    mask[idx] = True
    assert np.all(G.transpose(0, 2, 3, 1).reshape(-1, 9)[~mask] == 0)
    eps = 1e-6
    for k in [(0, 3, 0, 0), (0, 7, 0, 5), (1, 2, 1, 5)]:
        fp, fm = f.copy(), f.copy()
        fp[k] += eps
        fm[k] -= eps
        fd = (oracle.velocity_loss_subset(fp, idx, utx, uty)[0]
              - oracle.velocity_loss_subset(fm, idx, utx, uty)[0]) / (2 * eps)
        assert abs(fd - G[k]) <= 1e-7 * np.abs(G).max()
    t = f + inputs.noise(f.shape, 19, 0.01)
    Lp, Gp = oracle.population_loss_subset(f, idx, t)
    d = (f - t).transpose(0, 2, 3, 1).reshape(-1, 9)[idx]
    assert np.isclose(Lp, np.sum(d ** 2), rtol=1e-14)
    assert np.allclose(Gp.transpose(0, 2, 3, 1).reshape(-1, 9)[idx], 2 * d, rtol=1e-14)
    # zero at the target; a repeated node counts twice
    assert oracle.population_loss_subset(t, idx, t)[0] == 0.0
    L2, G2 = oracle.population_loss_subset(f, np.array([5, 5]), t)
    L1, G1 = oracle.population_loss_subset(f, np.array([5]), t)
    assert np.isclose(L2, 2 * L1, rtol=1e-15) and np.allclose(G2, 2 * G1, rtol=1e-15)


def test_subsample_is_strided_slice():
    f = inputs.noise((2, 9, 12, 16), 20, 1.0)
    assert np.array_equal(oracle.subsample(f, 4), f[:, :, ::4, ::4])

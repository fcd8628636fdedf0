"""Pins of the D3Q19 oracle (the paper's own 3D setting) against what the paper
and the mathematics fix, not against the oracle's own formulas:

* the stencil equals the paper's printed table (tests/golden/d3q19_stencil.txt);
* lattice quadrature up to fourth order, and the unweighted sums 19 and 10
  that the conservation layer's kappa denominators stand for;
* equilibrium moments (rho, rho u, rho u u + rho/3 I) exactly;
* streaming equals numpy.roll of every population; anti-streaming inverts it;
* BGK: mass and momentum conservation, equilibrium fixed point, and the shear
  viscosity nu = (tau - 1/2)/3 from the decay of shear waves along y and z;
* EDM forcing adds exactly F to the momentum; the force field has the
  printed structure (F_x(y), F_y(z), F_z(x)), zero mean, amplitude F;
* Smagorinsky: C_s = 0 is BGK; tau_eff solves the quadratic of the strain
  closure with Pi^neq computed here by einsum;
* the conservation layer equals the orthogonal projector onto the complement
  of span{1, c_x, c_y, c_z} computed by numpy least squares;
* the MLP equals a numpy restatement (LeakyReLU, slope 0.01); the learned
  collision is BGK for a zero output layer or an output in the conserved span;
* BGK and Smagorinsky steps commute with the cube's rotations and reflections.
"""
import os

import numpy as np
import pytest

import oracle.d3q19 as o3
from paper_2403_18466_gb300 import inputs

CX, CY, CZ, W = o3.lattice()
C = np.stack([CX, CY, CZ], 1)        # [19, 3]
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "d3q19_stencil.txt")


def _frac(s):
    a, b = s.split("/")
    return float(a) / float(b)


def test_stencil_is_the_papers_table():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    assert len(rows) == 19
    for r in rows:
        i = int(r[0])
        assert (CX[i], CY[i], CZ[i]) == (int(r[1]), int(r[2]), int(r[3]))
        assert W[i] == _frac(r[4])


def test_quadrature_and_unweighted_sums():
    d = np.eye(3)
    assert np.isclose(W.sum(), 1.0, rtol=0, atol=1e-16)
    assert np.allclose(np.einsum("i,ia->a", W, C), 0, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", W, C, C), d / 3, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib,ic->abc", W, C, C, C), 0, atol=1e-16)
    four = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
            + np.einsum("ad,bc->abcd", d, d)) / 9
    assert np.allclose(np.einsum("i,ia,ib,ic,id->abcd", W, C, C, C, C), four, atol=1e-16)
    # the plain sums behind kappa_1 = -1/19 sum, kappa_a = -1/10 sum c_a
    assert len(W) == 19 and np.array_equal(C.T @ C, 10 * np.eye(3, dtype=int))
    assert np.array_equal(C.sum(0), [0, 0, 0])
    # every velocity has its opposite
    for i in range(19):
        assert sum(np.array_equal(C[j], -C[i]) for j in range(19)) == 1


def test_equilibrium_moments():
    rng = np.random.default_rng(1)
    for _ in range(5):
        rho, u = 0.8 + 0.4 * rng.random(), 0.1 * rng.standard_normal(3)
        f = o3.feq(rho, u)
        assert np.isclose(f.sum(), rho, rtol=1e-15)
        assert np.allclose(C.T @ f, rho * u, rtol=0, atol=1e-15)
        P = np.einsum("i,ia,ib->ab", f, C, C)
        assert np.allclose(P, rho * np.outer(u, u) + rho / 3 * np.eye(3), rtol=0, atol=1e-15)


def _field(B, nz, ny, nx, seed, urms=0.04, neq=0.02):
    f = np.empty((B, 19, nz, ny, nx))
    for b in range(B):
        rho, u = inputs.random_velocity_field_3d(nz, ny, nx, seed=seed + b, k0=2.0, urms=urms)
        f[b] = o3.equilibrium_field(rho[None], u[None])[0]
    return f * (1 + inputs.noise(f.shape, seed + 100, neq))


def test_streaming_is_a_roll_and_antistreaming_inverts_it():
    g = _field(2, 5, 4, 6, 3)
    f = o3.stream_pull(g)
    for i in range(19):
        ref = np.roll(g[:, i], shift=(CZ[i], CY[i], CX[i]), axis=(1, 2, 3))
        assert np.array_equal(f[:, i], ref)
    assert np.array_equal(o3.stream_push(f), g)


def test_bgk_conserves_and_keeps_equilibrium():
    prm = o3.params(0.57)
    f = _field(1, 4, 5, 6, 7)[0, :, 1, 2, 3]
    post = o3.collide_node(o3.BGK, f, prm)
    assert np.isclose(post.sum(), f.sum(), rtol=1e-15)
    assert np.allclose(C.T @ post, C.T @ f, rtol=0, atol=1e-16)
    e = o3.feq(1.03, [0.02, -0.01, 0.015])
    assert np.allclose(o3.collide_node(o3.BGK, e, prm), e, rtol=0, atol=1e-16)


@pytest.mark.parametrize("axis", ["y", "z"])
def test_shear_wave_viscosity(axis):
    """u_x = u0 sin(k s), s = y or z, decays as exp(-nu k^2 t), nu = (tau - 1/2)/3."""
    tau, n, u0, T0, T1 = 0.6, 32, 1e-4, 20, 220
    k = 2 * np.pi / n
    nz, ny = (1, n) if axis == "y" else (n, 1)
    s = np.arange(n)
    u = np.zeros((1, 3, nz, ny, 1))
    if axis == "y":
        u[0, 0, 0, :, 0] = u0 * np.sin(k * s)
    else:
        u[0, 0, :, 0, 0] = u0 * np.sin(k * s)
    g = o3.stream_push(o3.equilibrium_field(np.ones((1, nz, ny, 1)), u))
    prm = o3.params(tau)
    amps = []
    for t in (T0, T1):
        gt = o3.run(o3.BGK, g, t, prm)
        _, v = o3.moments(o3.stream_pull(gt))
        prof = v[0, 0].reshape(-1)
        amps.append(2 / n * np.dot(prof, np.sin(k * s)))
    nu = np.log(amps[0] / amps[1]) / (k * k * (T1 - T0))
    assert abs(nu / ((tau - 0.5) / 3) - 1) < 0.02


def test_edm_force_and_force_field():
    rho, u, F = 1.05, np.array([0.01, -0.02, 0.005]), np.array([3e-4, -1e-4, 2e-4])
    fe = o3.edm_force(rho, u, F)
    assert abs(fe.sum()) < 1e-15 and np.allclose(C.T @ fe, F, rtol=1e-10, atol=0)
    prm = o3.params(0.6, force_amp=1e-3, force_mode=2)
    nz, ny, nx = 8, 6, 10
    Fs = np.array([[[o3.force(prm, z, y, x, nz, ny, nx) for x in range(nx)] for y in range(ny)]
                   for z in range(nz)])          # [nz, ny, nx, 3]
    assert np.allclose(Fs.mean(axis=(0, 1, 2)), 0, atol=1e-18)
    # F_x depends on y only, F_y on z only, F_z on x only
    assert np.allclose(Fs[..., 0], Fs[:1, :, :1, 0], rtol=0, atol=0)
    assert np.allclose(Fs[..., 1], Fs[:, :1, :1, 1], rtol=0, atol=0)
    assert np.allclose(Fs[..., 2], Fs[:1, :1, :, 2], rtol=0, atol=0)
    assert np.isclose(np.abs(Fs).max(), 1e-3, rtol=1e-12)
    # the force enters the collision as its EDM term
    f = _field(1, 3, 3, 3, 9)[0, :, 0, 0, 0]
    d = (o3.collide_node(o3.BGK, f, prm, F=F) - o3.collide_node(o3.BGK, f, prm))
    assert np.allclose(C.T @ d, F, rtol=1e-10, atol=0) and abs(d.sum()) < 1e-15


def test_smagorinsky_closure():
    f = _field(1, 3, 3, 3, 11, neq=0.05)[0, :, 1, 1, 1]
    prm0 = o3.params(0.52, smag_cs=0.0)
    assert np.array_equal(o3.collide_node(o3.SMAG, f, prm0), o3.collide_node(o3.BGK, f, prm0))
    rho = f.sum()
    u = C.T @ f / rho
    Pi = np.einsum("i,ia,ib->ab", f - o3.feq(rho, u), C, C)
    Q = np.sqrt(2 * np.sum(Pi * Pi))
    for tau0, cs in ((0.52, 0.1), (0.8, 0.3)):
        t = o3.smag_tau_eff(f, tau0, cs)
        assert t > tau0
        assert abs(t * t - tau0 * t - 9 * cs * cs * Q / (2 * rho)) < 1e-14


def test_projection_is_the_orthogonal_projector():
    V = np.stack([np.ones(19), CX, CY, CZ], 1).astype(float)
    P = np.eye(19) - V @ np.linalg.lstsq(V, np.eye(19), rcond=None)[0]
    rng = np.random.default_rng(4)
    for _ in range(4):
        o = rng.standard_normal(19)
        assert np.allclose(o3.project(o), P @ o, rtol=0, atol=1e-15)
    for v in V.T:
        assert np.allclose(o3.project(v), 0, atol=1e-15)


def _np_mlp(theta, x, widths, slope=0.01):
    dims = [19, *widths, 19]
    off, a = 0, np.asarray(x, float)
    for layer, (nin, nout) in enumerate(zip(dims[:-1], dims[1:])):
        Wl = theta[off:off + nin * nout].reshape(nout, nin)
        off += nin * nout
        bl = theta[off:off + nout]
        off += nout
        a = Wl @ a + bl
        if layer < len(dims) - 2:
            a = np.where(a >= 0, a, slope * a)
    assert off == len(theta)
    return a


@pytest.mark.parametrize("widths", [(300, 300, 100), (7, 5, 3)])
def test_mlp_matches_numpy_restatement(widths):
    theta = inputs.xavier_mlp_widths(5, widths, bias_scale=0.2, gain=2.0)
    assert len(theta) == o3.mlp_nparams(widths)
    prm = o3.params(0.6, widths=widths)
    x = np.random.default_rng(6).standard_normal(19) * 0.5
    out = o3.mlp_forward(theta, x, prm)
    assert np.allclose(out, _np_mlp(theta, x, widths), rtol=1e-13, atol=1e-15)
    # the negative branch really has slope 0.01 (not ReLU, not identity)
    ref0 = _np_mlp(theta, x, widths, slope=0.0)
    ref1 = _np_mlp(theta, x, widths, slope=1.0)
    assert not np.allclose(out, ref0) and not np.allclose(out, ref1)


def test_learned_collision_reductions_and_conservation():
    widths = (9, 8, 6)
    prm = o3.params(0.62, widths=widths)
    f = _field(1, 3, 3, 3, 13, neq=0.05)[0, :, 1, 2, 0]
    theta = inputs.xavier_mlp_widths(7, widths, bias_scale=0.3, gain=2.0)
    n_out = 19 * widths[-1] + 19
    zero_out = theta.copy()
    zero_out[-n_out:] = 0
    bgk = o3.collide_node(o3.BGK, f, prm)
    assert np.array_equal(o3.collide_node(o3.MLP, f, prm, zero_out), bgk)
    span = zero_out.copy()
    span[-19:] = 0.3 - 0.2 * CX + 0.1 * CZ       # output in span{1, c}
    assert np.allclose(o3.collide_node(o3.MLP, f, prm, span), bgk, rtol=0, atol=1e-15)
    post = o3.collide_node(o3.MLP, f, prm, theta)
    assert np.isclose(post.sum(), f.sum(), rtol=1e-15)
    assert np.allclose(C.T @ post, C.T @ f, rtol=0, atol=1e-16)
    assert not np.allclose(post, bgk)


def _rot(axis):
    c = {"z": [[0, -1, 0], [1, 0, 0], [0, 0, 1]], "x": [[1, 0, 0], [0, 0, -1], [0, 1, 0]],
         "mx": [[-1, 0, 0], [0, 1, 0], [0, 0, 1]], "swap": [[0, 1, 0], [1, 0, 0], [0, 0, 1]]}
    return np.array(c[axis])


def _transform(f, T):
    """(T f)_{pi(i)}(T x) = f_i(x), c_{pi(i)} = T c_i, on an n^3 periodic grid."""
    B, q, n, _, _ = f.shape
    out = np.empty_like(f)
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    X = np.stack([x, y, z])
    Xn = np.einsum("ab,bzyx->azyx", T, X) % n
    for i in range(19):
        j = [k for k in range(19) if np.array_equal(C[k], T @ C[i])][0]
        out[:, j, Xn[2], Xn[1], Xn[0]] = f[:, i, z, y, x]
    return out


@pytest.mark.parametrize("kind", [o3.BGK, o3.SMAG])
def test_step_commutes_with_cube_symmetries(kind):
    n = 6
    g = _field(1, n, n, n, 17, neq=0.03)
    prm = o3.params(0.53, smag_cs=0.3)
    ref = o3.run(kind, g, 2, prm)
    for name in ("z", "x", "mx", "swap"):
        T = _rot(name)
        a = o3.run(kind, _transform(g, T), 2, prm)
        assert np.allclose(a, _transform(ref, T), rtol=0, atol=1e-14 * np.abs(ref).max()), name
    # the transform itself: four quarter turns are the identity
    R = _rot("z")
    assert np.array_equal(_transform(_transform(_transform(_transform(g, R), R), R), R), g)

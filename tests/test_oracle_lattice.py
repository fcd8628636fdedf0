"""Pins of the oracle's lattice, equilibrium, streaming and parameter relations.

Each test checks the oracle against something the paper or the mathematics
fixes independently of the oracle's own code: quadrature identities of the
D2Q9 stencil, exact moments of the second-order equilibrium (Eq. S4), numbers
printed in Tab. S1, and streaming as a circular shift (numpy.roll).
"""
import os

import numpy as np
import pytest

import oracle
from paper_2403_18466_gb300 import inputs

CS2 = 1.0 / 3.0


def test_stencil_quadrature_identities():
    cx, cy, w = oracle.lattice()
    c = np.stack([cx, cy], 1).astype(float)
    assert np.isclose(w.sum(), 1.0, atol=1e-15)
    assert np.allclose(w @ c, 0.0, atol=1e-15)
    second = np.einsum("i,ia,ib->ab", w, c, c)
    assert np.allclose(second, CS2 * np.eye(2), atol=1e-15)
    third = np.einsum("i,ia,ib,ic->abc", w, c, c, c)
    assert np.allclose(third, 0.0, atol=1e-15)
    fourth = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    d = np.eye(2)
    iso = CS2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                      + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(fourth, iso, atol=1e-15)
    # every velocity has its opposite in the set; |c|^2 <= 2
    pairs = {(a, b) for a, b in zip(cx, cy)}
    assert all((-a, -b) in pairs for a, b in pairs)
    assert len(pairs) == 9 and max(cx ** 2 + cy ** 2) == 2
    # the projection denominators used for D2Q9: Q = 9 and sum c_a^2 = 6
    assert len(cx) == 9 and (cx ** 2).sum() == 6 and (cy ** 2).sum() == 6


@pytest.mark.parametrize("rho,ux,uy", [(1.0, 0.0, 0.0), (1.3, 0.05, -0.02), (0.7, -0.1, 0.08)])
def test_feq_moments_exact(rho, ux, uy):
    """Eq. S4 reproduces rho, rho u and rho uu + rho cs^2 I exactly."""
    cx, cy, w = oracle.lattice()
    c = np.stack([cx, cy], 1).astype(float)
    f = oracle.feq(rho, ux, uy)
    u = np.array([ux, uy])
    assert np.isclose(f.sum(), rho, rtol=0, atol=1e-15)
    assert np.allclose(f @ c, rho * u, rtol=0, atol=1e-15)
    P = np.einsum("i,ia,ib->ab", f, c, c)
    assert np.allclose(P, rho * np.outer(u, u) + rho * CS2 * np.eye(2), rtol=0, atol=1e-15)
    if ux == 0 and uy == 0:
        assert np.allclose(f, rho * w, rtol=0, atol=1e-16)


def _golden():
    here = os.path.join(os.path.dirname(__file__), "golden", "tab_s1.txt")
    vals = {}
    for line in open(here):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, v, sig = line.split()
        vals[name] = (float(v), int(sig))
    return vals


def _agrees(x, printed, sig):
    """x rounds to the printed value at the printed number of significant digits."""
    return float(f"{x:.{sig - 1}e}") == float(f"{printed:.{sig - 1}e}")


def test_tab_s1_viscosity_and_reynolds():
    """nu(tau) of Eq. S6 and Re = u_rms L / nu reproduce Tab. S1's printed values."""
    g = _golden()
    nu = oracle.viscosity(g["tau"][0])
    assert _agrees(nu, *g["nu"])
    Re = g["u_rms"][0] * g["L"][0] / nu
    assert _agrees(Re, *g["Re"])


def test_tau_rescaling_matches_printed_cg4():
    """Eq. S9 at cg = 4 gives the printed tau' = 0.5008; acoustic scaling keeps
    nu' cg = nu (dx and dt both grow by cg)."""
    g = _golden()
    tp = oracle.tau_rescaled(g["tau"][0], 4)
    assert _agrees(tp, *g["tau_prime_cg4"])
    for tau, cg in [(0.5032, 2), (0.503, 8), (0.6, 3)]:
        t2 = oracle.tau_rescaled(tau, cg)
        assert np.isclose(oracle.viscosity(t2) * cg, oracle.viscosity(tau), rtol=1e-14)
    assert np.isclose(oracle.tau_rescaled(0.503, 8), 0.500375, rtol=0, atol=1e-15)


def _rand_field(B, ny, nx, seed):
    return 0.1 + inputs.noise((B, 9, ny, nx), seed, 0.05)


def test_stream_pull_is_circular_shift():
    cx, cy, _ = oracle.lattice()
    g = _rand_field(2, 7, 11, 1)
    f = oracle.stream_pull(g)
    for i in range(9):
        ref = np.roll(g[:, i], shift=(cy[i], cx[i]), axis=(1, 2))
        assert np.array_equal(f[:, i], ref)


def test_stream_push_inverts_pull_and_preserves_sums():
    g = _rand_field(1, 9, 6, 2)
    f = oracle.stream_pull(g)
    assert np.array_equal(oracle.stream_push(f), g)
    assert np.array_equal(oracle.stream_pull(oracle.stream_push(g)), g)
    # a permutation: the multiset of values per plane is unchanged
    for i in range(9):
        assert np.array_equal(np.sort(f[0, i].ravel()), np.sort(g[0, i].ravel()))


def test_repeated_streaming_is_shift_by_n_c():
    cx, cy, _ = oracle.lattice()
    g = _rand_field(1, 8, 10, 3)
    f = g.copy()
    n = 13
    for _ in range(n):
        f = oracle.stream_pull(f)
    for i in range(9):
        assert np.array_equal(f[0, i], np.roll(g[0, i], (n * cy[i], n * cx[i]), axis=(0, 1)))


def test_moments_against_direct_sums():
    cx, cy, _ = oracle.lattice()
    f = _rand_field(2, 5, 4, 4)
    rho, ux, uy = oracle.moments(f)
    assert np.allclose(rho, f.sum(1), rtol=1e-15)
    assert np.allclose(ux, np.einsum("bixy,i->bxy", f, cx) / f.sum(1), rtol=1e-14)
    assert np.allclose(uy, np.einsum("bixy,i->bxy", f, cy) / f.sum(1), rtol=1e-14)

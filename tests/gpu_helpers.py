"""Shared helpers of the GPU parity tests (test code, not library code)."""
import numpy as np

import oracle
from paper_2403_18466_gb300 import inputs


def population_field(B, ny, nx, seed, urms=0.03, neq=0.01, k0=3.0, mean_u=(0.01, -0.005)):
    """Seeded FP32 pre-collision populations: feq of a random divergence-free
    field (per lattice) plus a uniform mean flow, with a small multiplicative
    non-equilibrium part.  The mean flow keeps |u| away from zero on tiny
    grids, so relative velocity errors stay well conditioned.  Built with the
    oracle's equilibrium (test inputs may come from the oracle)."""
    out = np.empty((B, 9, ny, nx))
    for b in range(B):
        rho, ux, uy = inputs.random_velocity_field(ny, nx, seed=seed + b, k0=k0, urms=urms)
        ux = ux + mean_u[0]
        uy = uy + mean_u[1]
        rho = rho * (1.0 + inputs.noise(rho.shape, seed + 100 + b, 0.01))
        out[b] = oracle.equilibrium_field(rho[None], ux[None], uy[None])[0]
    out *= 1.0 + inputs.noise(out.shape, seed + 200, neq)
    return out.astype(np.float32)


def rel_pop_err(a, ref):
    """max_{i,x} |a - ref| / |ref| (populations are positive)."""
    return float(np.max(np.abs(a - ref) / np.abs(ref)))


def weighted_pop_err(a, ref):
    """max_{i,x} |a - ref| / w_i: population error on the scale of each
    population's weight (well conditioned where a population nears zero)."""
    _, _, w = oracle.lattice()
    return float(np.max(np.abs(a - ref) / w[None, :, None, None]))


def rel_vel_err(ux, uy, rx, ry):
    """||u - u_ref||_inf / ||u_ref||_inf over both components."""
    num = max(np.abs(ux - rx).max(), np.abs(uy - ry).max())
    den = max(np.abs(rx).max(), np.abs(ry).max())
    return float(num / den)


def bf16_round(a):
    """Round float64 values to bfloat16 (round to nearest even), returned as float64."""
    import torch
    return torch.tensor(np.asarray(a, dtype=np.float64)).to(torch.bfloat16).double().numpy()


def learned_pop_check(got, ref, ref_bgk, alpha):
    """Population-level parity of a learned-collision result.

    got, ref, ref_bgk: post-collision populations (same shape, [..., 9, ...] with
    the population index on axis -3, or [n, 9] rows).  The error and the learned
    correction are measured on the scale of each population's weight w_i:
      err  = max |got - ref| / w_i,   corr = max |ref - ref_bgk| / w_i,
    and the check passes when err <= alpha * corr.  A result without the learned
    part (plain BGK) has err = corr and fails for any alpha < 1.
    Returns (ok, err, corr, tol)."""
    _, _, w = oracle.lattice()
    got, ref, ref_bgk = (np.asarray(a, dtype=np.float64) for a in (got, ref, ref_bgk))
    ws = w[:, None, None] if got.ndim >= 3 else w[None, :]
    err = float(np.max(np.abs(got - ref) / ws))
    corr = float(np.max(np.abs(ref - ref_bgk) / ws))
    tol = alpha * corr
    return err <= tol, err, corr, tol


def post_collision(lat):
    """Post-collision populations g = state + w_i of a Lattice, as float64 numpy
    [b][i][y][x] (the stored state is g - w_i)."""
    _, _, w = oracle.lattice()
    return lat.state_tensor().double().cpu().numpy() + w[None, :, None, None]


def learned_theta(seed=5, in_scale=30.0, out_scale=0.0025):
    """Test weights of the 9 -> 64 -> 64 -> 9 network that exercise every part of
    the learned collision: hidden layers with Xavier gain 3 and biases of +-0.3
    (saturating tanh), a first layer scaled by `in_scale` so that the inputs
    x = (f - feq)/rho (~1e-2) drive the hidden units about as much as the
    biases do, and an output layer scaled by `out_scale` so that one step moves
    the velocity by a few per cent (several times the 2e-3 velocity tolerance,
    small enough that the bf16 error stays inside it)."""
    theta = inputs.xavier_mlp(seed, bias_scale=0.3, gain=3.0, out_scale=out_scale)
    inputs.unpack_mlp(theta)[0][:] *= in_scale
    return theta

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

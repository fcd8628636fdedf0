"""Training data the method generates itself (SI section 2, "Definition of the
Training Dataset"), with a box average (default) or the paper's subsampling as
the coarse-graining filter phi.

1. Fine-grid DNS: BGK at tau on an n x n periodic grid under Kolmogorov
   forcing F_x = F0 sin(2 pi m y / n), from a random-phase divergence-free
   initial field, run on the GPU (``lbm_step(LBM_BGK)``).
2. After a spin-up, snapshots every ``stride`` fine steps.  Each snapshot gives
   one trajectory: the box-filtered pre-collision populations at the snapshot
   (``lbm_box_filter``, cg x cg blocks, or ``lbm_subsample``) are the coarse
   initial state, and the filtered state after ``cg * unroll`` fine steps (one
   coarse step is cg fine steps) gives the targets of the unrolled loss: its
   velocity, and its populations anti-streamed on the coarse grid
   (``lbm_stream``, direction -1), which are the post-collision populations
   the last unrolled step must produce (SI section 2, steps 1-4).
3. Coarse-grid parameters: tau' = (tau - 1/2)/cg + 1/2 (Eq. S9); under
   acoustic scaling the body force per unit mass becomes F' = cg * F0 with
   the same mode number m.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import inputs, lbm


@dataclass
class Dataset:
    f0: torch.Tensor      # [B, 9, N, N] coarse pre-collision populations
    utx: torch.Tensor     # [B, N, N] target velocity after `unroll` coarse steps
    uty: torch.Tensor
    target_post: torch.Tensor  # [B, 9, N, N] post-collision populations of the last step
    tau_les: float
    force_les: float
    force_mode: int
    unroll: int
    cg: int


def rescaled_tau(tau, cg):
    """Eq. S9."""
    return (tau - 0.5) / cg + 0.5


def generate(n=2048, cg=8, tau=0.503, force_amp=1e-5, force_mode=4, trajectories=32,
             unroll=16, spinup=5000, stride=200, seed=4, k0=8.0, urms=0.02, device="cuda",
             filter="box"):
    """Run the DNS and cut `trajectories` (initial state, targets) tuples.
    filter: "box" (cg x cg block mean) or "subsample" (the paper's phi)."""
    if filter not in ("box", "subsample"):
        raise ValueError(f"unknown filter {filter!r}")
    rho, ux, uy = inputs.random_velocity_field(n, n, seed=seed, k0=k0, urms=urms)
    dns = lbm.Lattice(n, n, 1, tau=tau, force_amp=force_amp, force_mode=force_mode, device=device)
    t = lambda a: torch.tensor(a[None], dtype=torch.float32, device=device)
    dns.init_equilibrium(t(rho), t(ux), t(uy))
    dns.step(spinup, "bgk")
    N = n // cg
    f0 = torch.empty((trajectories, 9, N, N), dtype=torch.float32, device=device)
    utx = torch.empty((trajectories, N, N), dtype=torch.float32, device=device)
    uty = torch.empty_like(utx)
    target_post = torch.empty_like(f0)
    tmp = lbm.Lattice(N, N, 1, tau=rescaled_tau(tau, cg), device=device)
    phi = dns.box_filter if filter == "box" else dns.subsample
    horizon = cg * unroll
    for k in range(trajectories):
        phi(cg, out=f0[k:k + 1])
        dns.step(horizon, "bgk")
        fc = phi(cg)
        tmp.set_state(fc)
        _, vx, vy = tmp.moments()
        utx[k], uty[k] = vx[0], vy[0]
        tmp.stream(fc, -1, out=target_post[k:k + 1])
        if stride > horizon:
            dns.step(stride - horizon, "bgk")
    if dns.status() != lbm.LBM_OK:
        raise RuntimeError(f"DNS became unstable: {lbm.lbm_strerror(dns.status())}")
    return Dataset(f0, utx, uty, target_post, rescaled_tau(tau, cg), cg * force_amp, force_mode,
                   unroll, cg)

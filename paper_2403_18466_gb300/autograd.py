"""Unrolled learned-collision lattice Boltzmann as a ``torch.autograd.Function``.

Forward (SI section 2, "Unrolled training"): load the pre-collision
populations f0, advance ``nsteps`` steps with the FP32 learned collision while
recording a checkpoint every ``ckpt_every`` steps (``lbm_forward_record``), and
return the loss at the final step: the velocity loss on every node
(``lbm_velocity_loss``), or a loss on a node subset S, either its velocity form
(``lbm_velocity_loss_subset``) or the population form of Eq. S13 on the
post-collision populations of the last step (``lbm_population_loss_subset``).
Backward: the library's hand-written adjoint (``lbm_backward``) recomputes
each segment from its checkpoint and returns dL/dtheta (and dL/df0).

Every operation runs in the C ABI's kernels; this module only passes device
pointers.  The weights are the packed parameter vector of the library
(w1[64][9], b1, w2[64][64], b2, w3[9][64], b3; LBM_MLP_NPARAMS floats).
"""
from __future__ import annotations

import torch

from . import lbm


class UnrolledLBM:
    """Owns the lattice and the checkpoint workspace of one unroll shape."""

    def __init__(self, nx, ny, batch, tau, nsteps, ckpt_every=4, force_amp=0.0, force_mode=0,
                 device="cuda", precision="f32"):
        """precision "f32": FP32 learned collision and FP32 CUDA-core adjoint;
        "bf16": tensor-core learned collision and tensor-core adjoint."""
        assert precision in ("f32", "bf16")
        self.precision = precision
        self.lat = lbm.Lattice(nx, ny, batch, tau=tau, force_amp=force_amp,
                               force_mode=force_mode, device=device)
        self.nsteps, self.ckpt_every = int(nsteps), int(ckpt_every)
        nbytes = self.lat.record_bytes(self.nsteps, self.ckpt_every)
        self.ws = torch.empty(nbytes // 4, dtype=torch.float32, device=device)
        self.dW = torch.empty(lbm.LBM_MLP_NPARAMS, dtype=torch.float32, device=device)

    def loss(self, theta, f0, utx, uty):
        """Differentiable velocity loss of the unroll (w.r.t. theta and f0)."""
        return _UnrollFn.apply(theta, f0, self, ("velocity", None, utx, uty))

    def loss_subset(self, theta, f0, idx, utx=None, uty=None, target_post=None):
        """Differentiable loss on the nodes idx (int32 device tensor of flat
        indices b*N*N + y*N + x): the velocity form against (utx, uty), or,
        with target_post, Eq. S13 against target post-collision populations."""
        if target_post is not None:
            return _UnrollFn.apply(theta, f0, self, ("population", idx, target_post, None))
        return _UnrollFn.apply(theta, f0, self, ("velocity_subset", idx, utx, uty))


def _final_loss(lat, spec):
    form, idx, a, b = spec
    if form == "velocity":
        return lat.velocity_loss(a.contiguous(), b.contiguous(), want_grad=True)
    if form == "velocity_subset":
        return lat.velocity_loss_subset(idx, a.contiguous(), b.contiguous(), want_grad=True)
    return lat.population_loss_subset(idx, a.contiguous(), want_grad=True)


class _UnrollFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, f0, run: UnrolledLBM, spec):
        theta_c = theta.detach().contiguous()
        w = lbm.weights_struct(theta_c)
        lat = run.lat
        lat.set_state(f0.detach().contiguous())
        lat.forward_record(run.nsteps, run.ckpt_every, w, run.ws, run.precision)
        loss, dL_df = _final_loss(lat, spec)
        ctx.run, ctx.w, ctx.theta = run, w, theta_c
        ctx.save_for_backward(dL_df)
        ctx.want_f0 = f0.requires_grad
        return loss[0].clone()

    @staticmethod
    def backward(ctx, grad_out):
        (dL_df,) = ctx.saved_tensors
        run = ctx.run
        df0 = torch.empty_like(dL_df) if ctx.want_f0 else None
        run.lat.backward(dL_df, ctx.w, run.ws, run.dW, df0, run.precision)
        g_theta = run.dW.clone() * grad_out
        g_f0 = df0 * grad_out if df0 is not None else None
        return g_theta, g_f0, None, None

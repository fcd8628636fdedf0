"""Unrolled training of the collision MLP (SI section 2, "Unrolled training").

Each epoch: evolve every training trajectory for `unroll` coarse steps with the
learned collision, compute the loss at the final step (velocity loss on every
node by default; with ``subset`` > 0, a fresh random node subset S per epoch
and either the velocity form or the population form of Eq. S13), backpropagate
through all steps with the library's hand-written adjoint (tensor-core pair by
default, FP32 CUDA-core pair on request), and take an Adam step (learning rate 1e-4, weight decay 1e-6, Tab. S1).  Plain BGK and
Smagorinsky-BGK LES from the same initial states are evaluated with the same
loss as the baselines the learned collision is compared with.

    python -m paper_2403_18466_gb300.train --epochs 200
"""
from __future__ import annotations

import argparse
import json
import time

import torch

from . import data as data_mod
from . import inputs, lbm
from .autograd import UnrolledLBM


def rollout_loss(ds, kind, theta=None, smag_cs=0.1):
    """Velocity loss of a plain (non-differentiated) LES rollout of `kind`."""
    B, _, N, _ = ds.f0.shape
    lat = lbm.Lattice(N, N, B, tau=ds.tau_les, smag_cs=smag_cs, force_amp=ds.force_les,
                      force_mode=ds.force_mode, device=ds.f0.device)
    lat.set_state(ds.f0)
    w = lbm.weights_struct(theta.detach().contiguous()) if theta is not None else None
    lat.step(ds.unroll, kind, w)
    loss, _ = lat.velocity_loss(ds.utx, ds.uty, want_grad=False)
    return float(loss.item()), lat.status()


def subset_indices(nodes, size, gen, device):
    """A random subset S of `size` distinct flat node indices (int32)."""
    return torch.randperm(nodes, generator=gen)[:size].to(device=device, dtype=torch.int32)


def train(ds, epochs=200, lr=1e-4, weight_decay=1e-6, ckpt_every=4, seed=3, out_scale=0.01,
          log_every=10, verbose=True, precision="bf16", subset=0, loss="velocity"):
    """precision "bf16": tensor-core forward and adjoint; "f32": CUDA-core FP32 pair.
    subset > 0 draws |S| = subset nodes per epoch (the paper uses 512);
    loss "velocity" or "population" (Eq. S13, needs subset > 0)."""
    if loss not in ("velocity", "population") or (loss == "population" and subset <= 0):
        raise ValueError("loss must be 'velocity', or 'population' with subset > 0")
    dev = ds.f0.device
    B, _, N, _ = ds.f0.shape
    theta = torch.nn.Parameter(torch.tensor(inputs.xavier_mlp(seed, out_scale=out_scale),
                                            dtype=torch.float32, device=dev))
    opt = torch.optim.Adam([theta], lr=lr, weight_decay=weight_decay)
    run = UnrolledLBM(N, N, B, ds.tau_les, ds.unroll, ckpt_every, ds.force_les, ds.force_mode,
                      device=dev, precision=precision)
    gen = torch.Generator().manual_seed(seed)
    history = []
    t0 = time.perf_counter()
    for ep in range(epochs):
        opt.zero_grad(set_to_none=True)
        if subset > 0:
            idx = subset_indices(B * N * N, subset, gen, dev)
            if loss == "population":
                L = run.loss_subset(theta, ds.f0, idx, target_post=ds.target_post)
            else:
                L = run.loss_subset(theta, ds.f0, idx, ds.utx, ds.uty)
        else:
            L = run.loss(theta, ds.f0, ds.utx, ds.uty)
        L.backward()
        opt.step()
        history.append(float(L.item()))
        if verbose and (ep % log_every == 0 or ep == epochs - 1):
            print(json.dumps({"epoch": ep, "loss": history[-1],
                              "elapsed_s": round(time.perf_counter() - t0, 2)}), flush=True)
    return theta.detach(), history


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--dns", type=int, default=2048)
    ap.add_argument("--cg", type=int, default=8)
    ap.add_argument("--trajectories", type=int, default=32)
    ap.add_argument("--unroll", type=int, default=16)
    ap.add_argument("--epochs", type=int, default=200)
    ap.add_argument("--lr", type=float, default=1e-4)
    ap.add_argument("--precision", default="bf16", choices=["bf16", "f32"])
    ap.add_argument("--filter", default="box", choices=["box", "subsample"])
    ap.add_argument("--subset", type=int, default=0, help="|S| of the subset loss (paper: 512)")
    ap.add_argument("--loss", default="velocity", choices=["velocity", "population"])
    ap.add_argument("--save", default=None, help="write the trained weights (.npy: float32 packed vector)")
    args = ap.parse_args()
    ds = data_mod.generate(n=args.dns, cg=args.cg, trajectories=args.trajectories,
                           unroll=args.unroll, filter=args.filter)
    base = {k: rollout_loss(ds, k)[0] for k in ("bgk", "smag")}
    print(json.dumps({"baseline_loss": base}), flush=True)
    theta, hist = train(ds, epochs=args.epochs, lr=args.lr, precision=args.precision,
                        subset=args.subset, loss=args.loss)
    learned = rollout_loss(ds, "mlp_bf16" if args.precision == "bf16" else "mlp_f32", theta)[0]
    print(json.dumps({"trained_loss": learned, "first_epoch_loss": hist[0],
                      "baseline_loss": base}), flush=True)
    if args.save:
        inputs.save_weights(theta, args.save)


if __name__ == "__main__":
    main()

"""A-posteriori evaluation of the learned collision against the filtered DNS
(main text: LES with the learned collision compared with plain BGK and
Smagorinsky LES and with the filtered DNS through energy spectra and structure
functions).

1. Generate training data from a fine-grid DNS (``data.generate``) and train
   the collision (``train.train``, tensor-core pair by default).
2. From a later DNS state, start the coarse LES runs (BGK, Smagorinsky,
   learned) on the filtered populations and advance the DNS alongside (cg fine
   steps per coarse step).
3. Every ``every`` coarse steps record E(k) and S^p(r) of each LES and of the
   filtered DNS; report the relative L2 error of each LES spectrum against the
   filtered DNS over the resolved shells, and the velocity error.  A run whose
   status turns unstable is stopped and reported (plain BGK at the coarse
   parameters is expected to be, as the paper notes).

    python -m paper_2403_18466_gb300.evaluate --dns 2048 --cg 8 --epochs 200 --steps 2000
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import data as data_mod
from . import inputs, lbm
from .train import train


def _spectrum_error(E, Eref, kmax):
    k = slice(1, kmax + 1)
    return float(np.linalg.norm(E[k] - Eref[k]) / np.linalg.norm(Eref[k]))


def evaluate(dns=2048, cg=8, tau=0.503, force_amp=1e-5, force_mode=4, epochs=200, lr=1e-3,
             trajectories=32, unroll=16, steps=2000, every=250, spinup=5000, seed=4,
             precision="bf16", smag_cs=0.1, filter="box", device="cuda", verbose=True,
             dns_eval=None, theta=None):
    """dns_eval: size of the evaluation DNS (default: the training DNS size);
    the learned collision is local, so a model trained on the dns -> dns/cg
    pair applies to any dns_eval -> dns_eval/cg pair at the same tau and cg.
    theta: trained weights to use instead of training here."""
    t0 = time.perf_counter()
    hist = [float("nan")]
    if theta is None:
        ds = data_mod.generate(n=dns, cg=cg, tau=tau, force_amp=force_amp,
                               force_mode=force_mode, trajectories=trajectories, unroll=unroll,
                               spinup=spinup, seed=seed, filter=filter, device=device)
        theta, hist = train(ds, epochs=epochs, lr=lr, verbose=False, precision=precision)
    t_train = time.perf_counter() - t0

    # a fresh DNS state beyond the training snapshots, and its filtered populations
    n = dns_eval or dns
    N = n // cg
    rho, ux, uy = inputs.random_velocity_field(n, n, seed=seed + 100, k0=8.0, urms=0.02)
    fine = lbm.Lattice(n, n, 1, tau=tau, force_amp=force_amp, force_mode=force_mode,
                       device=device)
    t = lambda a: torch.tensor(a[None], dtype=torch.float32, device=device)
    fine.init_equilibrium(t(rho), t(ux), t(uy))
    fine.step(spinup, "bgk")
    phi = fine.box_filter if filter == "box" else fine.subsample
    f0 = phi(cg)
    runs = {}
    w = lbm.weights_struct(theta.contiguous())
    kind_learned = "mlp_bf16" if precision == "bf16" else "mlp_f32"
    tau_les, force_les = data_mod.rescaled_tau(tau, cg), cg * force_amp
    for name, kind in (("bgk", "bgk"), ("smag", "smag"), ("learned", kind_learned)):
        lat = lbm.Lattice(N, N, 1, tau=tau_les, smag_cs=smag_cs, force_amp=force_les,
                          force_mode=force_mode, device=device)
        lat.set_state(f0)
        runs[name] = (lat, kind)
    ref = lbm.Lattice(N, N, 1, tau=tau_les, device=device)  # holds the filtered DNS state
    kmax = N // 2
    rmax = N // 4
    out = {"steps": [], "spectrum_error": {k: [] for k in runs}, "velocity_error": {k: [] for k in runs},
           "energy": {k: [] for k in list(runs) + ["dns"]}, "status": {}}
    E_last, S_last = {}, {}
    alive = {name: True for name in runs}
    out["unstable_at"] = {name: None for name in runs}
    done = 0
    while done < steps:
        k = min(every, steps - done)
        fine.step(cg * k, "bgk")
        for name, (lat, kind) in runs.items():
            if alive[name]:
                lat.step(k, kind, w if kind.startswith("mlp") else None)
        done += k
        ref.set_state(phi(cg))
        Eref = ref.energy_spectrum(kmax).cpu().numpy()
        _, vx, vy = ref.moments()
        out["steps"].append(done)
        out["energy"]["dns"].append(float(Eref.sum()))
        E_last["dns"], S_last["dns"] = Eref, ref.structure_functions(rmax).cpu().numpy()
        for name, (lat, kind) in runs.items():
            if alive[name] and lat.status() != lbm.LBM_OK:
                # coarse plain LBM at these parameters is expected to blow up (SI section 2)
                alive[name] = False
                out["unstable_at"][name] = done
            if not alive[name]:
                out["spectrum_error"][name].append(float("nan"))
                out["velocity_error"][name].append(float("nan"))
                out["energy"][name].append(float("nan"))
                continue
            E = lat.energy_spectrum(kmax).cpu().numpy()
            _, lx, ly = lat.moments()
            out["spectrum_error"][name].append(_spectrum_error(E, Eref, kmax // 2))
            verr = torch.sqrt(((lx - vx) ** 2 + (ly - vy) ** 2).mean() / (vx ** 2 + vy ** 2).mean())
            out["velocity_error"][name].append(float(verr))
            out["energy"][name].append(float(E.sum()))
            E_last[name], S_last[name] = E, lat.structure_functions(rmax).cpu().numpy()
        if verbose:
            print(json.dumps({"step": done, **{f"E_err_{k}": round(v[-1], 4)
                                               for k, v in out["spectrum_error"].items()}}),
                  flush=True)
    for name, (lat, _) in runs.items():
        out["status"][name] = lbm.lbm_strerror(lat.status())
    out["train"] = {"epochs": epochs, "first_loss": hist[0], "last_loss": hist[-1],
                    "seconds": round(t_train, 1)}
    out["pair"] = {"dns": n, "les": N, "cg": cg, "tau_les": tau_les, "force_les": force_les}
    if fine.status() != lbm.LBM_OK:
        out["dns_status"] = lbm.lbm_strerror(fine.status())
    out["wall_s"] = round(time.perf_counter() - t0, 1)
    out["final_spectra"] = {k: v.tolist() for k, v in E_last.items()}
    out["final_S2"] = {k: v[1].tolist() for k, v in S_last.items()}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--dns", type=int, default=2048)
    ap.add_argument("--cg", type=int, default=8)
    ap.add_argument("--epochs", type=int, default=200)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--every", type=int, default=250)
    ap.add_argument("--precision", default="bf16", choices=["bf16", "f32"])
    ap.add_argument("--filter", default="box", choices=["box", "subsample"])
    ap.add_argument("--out", default=None, help="write the full record as JSON")
    ap.add_argument("--dns-eval", type=int, default=None, help="evaluation DNS size")
    ap.add_argument("--weights", default=None, help="trained weights (torch.save), skip training")
    args = ap.parse_args()
    theta = inputs.load_weights(args.weights, "cuda") if args.weights else None
    res = evaluate(dns=args.dns, cg=args.cg, epochs=args.epochs, lr=args.lr, steps=args.steps,
                   every=args.every, precision=args.precision, filter=args.filter,
                   dns_eval=args.dns_eval, theta=theta)
    summary = {k: res[k] for k in ("steps", "spectrum_error", "velocity_error", "status",
                                   "unstable_at", "train", "wall_s", "pair")}
    print(json.dumps(summary))
    if args.out:
        with open(args.out, "w") as fh:
            json.dump(res, fh)


if __name__ == "__main__":
    main()

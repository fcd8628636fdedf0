"""Long LES runs with on-device turbulence statistics (main-text energy spectra,
SI section 3 structure functions and extended self-similarity).

``run`` advances one lattice with a chosen collision and records, every
``every`` steps, the energy spectrum E(k) and the longitudinal structure
functions S^p(r), p = 1..6; ``ess_exponents`` turns averaged structure
functions into extended-self-similarity exponents xi_p / xi_3 (slopes of
log |S^p| against log |S^3| over a chosen range of S^3).

    python -m paper_2403_18466_gb300.les --n 1024 --kind smag --steps 10000 --every 1000
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import inputs, lbm


def run(n=1024, kind="smag", steps=10000, every=1000, tau=0.51, smag_cs=0.1, force_amp=1e-5,
        force_mode=4, seed=1, k0=8.0, urms=0.02, theta=None, rmax=None, kmax=None,
        device="cuda"):
    """Returns dict with step list, spectra [m, kmax+1], structure functions
    [m, 6, rmax] (numpy), the wall time, and the lattice status."""
    rho, ux, uy = inputs.random_velocity_field(n, n, seed=seed, k0=k0, urms=urms)
    lat = lbm.Lattice(n, n, 1, tau=tau, smag_cs=smag_cs, force_amp=force_amp,
                      force_mode=force_mode, device=device)
    t = lambda a: torch.tensor(a[None], dtype=torch.float32, device=device)
    lat.init_equilibrium(t(rho), t(ux), t(uy))
    w = lbm.weights_struct(theta.contiguous()) if theta is not None else None
    rmax = rmax or n // 4
    kmax = kmax or n // 2
    steps_rec, spectra, sfs = [], [], []
    t0 = time.perf_counter()
    done = 0
    while done < steps:
        k = min(every, steps - done)
        lat.step(k, kind, w)
        done += k
        spectra.append(lat.energy_spectrum(kmax))
        sfs.append(lat.structure_functions(rmax))
        steps_rec.append(done)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    return {"steps": steps_rec, "E": torch.stack(spectra).cpu().numpy(),
            "S": torch.stack(sfs).cpu().numpy(), "wall_s": wall,
            "mlups": n * n * steps / wall / 1e6, "status": lbm.lbm_strerror(lat.status())}


def ess_exponents(S, s3_range=None):
    """Extended self-similarity: for each p, the least-squares slope of
    log |S^p(r)| against log |S^3(r)| over the r where |S^3| lies in s3_range
    (default: all r).  S is [6, rmax] (row p-1 = S^p).  Returns slopes for
    p = 1..6 (the slope for p = 3 is 1 by construction)."""
    S = np.asarray(S, dtype=np.float64)
    s3 = np.abs(S[2])
    sel = np.ones_like(s3, dtype=bool) if s3_range is None else (s3 >= s3_range[0]) & (s3 <= s3_range[1])
    sel &= s3 > 0
    if sel.sum() < 2:
        return np.full(6, np.nan)
    x = np.log(s3[sel])
    out = []
    for p in range(6):
        y = np.log(np.abs(S[p][sel]) + 1e-300)
        out.append(np.polyfit(x, y, 1)[0])
    return np.array(out)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--kind", default="smag", choices=["bgk", "smag", "mlp_bf16", "mlp_f32"])
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--every", type=int, default=1000)
    ap.add_argument("--tau", type=float, default=0.51)
    ap.add_argument("--weights", default=None, help="torch.save'd packed weights (MLP kinds)")
    args = ap.parse_args()
    theta = None
    if args.weights:
        theta = torch.load(args.weights).to("cuda", torch.float32)
    res = run(n=args.n, kind=args.kind, steps=args.steps, every=args.every, tau=args.tau,
              theta=theta)
    S_mean = res["S"].mean(0)
    print(json.dumps({"kind": args.kind, "n": args.n, "steps": args.steps,
                      "mlups": round(res["mlups"], 1), "status": res["status"],
                      "energy": float(res["E"][-1].sum()),
                      "ess": [round(float(v), 4) for v in ess_exponents(S_mean)]}))


if __name__ == "__main__":
    main()

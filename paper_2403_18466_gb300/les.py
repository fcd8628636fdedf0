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
        device="cuda", stop_on_unstable=False, check_every=None):
    """Returns dict with step list, spectra [m, kmax+1], structure functions
    [m, 6, rmax] (numpy), the wall time, and the lattice status.  With
    stop_on_unstable, the run ends at the first record whose status is not OK
    (|u| >= 0.4 or non-finite somewhere since the previous record) and
    "unstable_at" gives that record's step (None if it stayed stable); with
    check_every (a divisor of every) the status is also read every
    check_every steps, so unstable_at is known to that resolution."""
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
    unstable_at = None
    step_time = 0.0
    while done < steps:
        k = min(every, steps - done)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sub = check_every if (stop_on_unstable and check_every) else k
        a.record()
        left = k
        while left > 0:
            lat.step(min(sub, left), kind, w)
            done += min(sub, left)
            left -= min(sub, left)
            if stop_on_unstable and left > 0 and lat.status() != lbm.LBM_OK:
                unstable_at = done
                break
        b.record()
        b.synchronize()
        if unstable_at is None and stop_on_unstable and lat.status() != lbm.LBM_OK:
            unstable_at = done
        if unstable_at is not None:
            break
        step_time += a.elapsed_time(b) * 1e-3
        spectra.append(lat.energy_spectrum(kmax))
        sfs.append(lat.structure_functions(rmax))
        steps_rec.append(done)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    stepped = steps_rec[-1] if steps_rec else 0
    return {"steps": steps_rec,
            "E": torch.stack(spectra).cpu().numpy() if spectra else np.zeros((0, kmax + 1)),
            "S": torch.stack(sfs).cpu().numpy() if sfs else np.zeros((0, 6, rmax)),
            "wall_s": wall, "unstable_at": unstable_at,
            "mlups": n * n * stepped / step_time / 1e6 if step_time > 0 else float("nan"),
            "status": lbm.lbm_strerror(lat.status())}


def long_comparison(theta, n=8192, steps=100000, every=1000, tau=0.500375, smag_cs=0.1,
                    force_amp=1e-5, force_mode=4, seed=5, rmax=256, device="cuda",
                    check_every=100):
    """The long learned-collision LES against the Smagorinsky LES from the same
    initial field: each run until `steps` or its first unstable record.
    Returns, per kind, the records' steps and energies, the spectrum and
    S^p(r) (p = 2..6, r = 1..rmax) at the last stable record and every tenth
    record, the ESS exponents of the time-averaged S^p, the unstable step and
    the throughput of the stepping."""
    out = {}
    for kind in ("mlp_bf16", "smag"):
        res = run(n=n, kind=kind, steps=steps, every=every, tau=tau, smag_cs=smag_cs,
                  force_amp=force_amp, force_mode=force_mode, seed=seed,
                  theta=theta if kind == "mlp_bf16" else None, rmax=rmax, device=device,
                  stop_on_unstable=True, check_every=check_every)
        E, S = res["E"], res["S"]
        keep = list(range(0, len(res["steps"]), 10)) + ([len(res["steps"]) - 1] if len(res["steps"]) else [])
        out[kind] = {
            "steps": res["steps"], "energy": [float(e.sum()) for e in E],
            "unstable_at": res["unstable_at"], "mlups": round(res["mlups"], 1),
            "wall_s": round(res["wall_s"], 1),
            "spectra": {int(res["steps"][i]): E[i].tolist() for i in sorted(set(keep))},
            "S": {int(res["steps"][i]): S[i][1:].tolist() for i in sorted(set(keep))},
            "ess": [float(v) for v in ess_exponents(S.mean(0))] if len(S) else None,
        }
    return out


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
    ap.add_argument("--compare", action="store_true",
                    help="learned (--weights) against Smagorinsky, until unstable")
    ap.add_argument("--out", default=None, help="write the comparison record as JSON")
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--kind", default="smag", choices=["bgk", "smag", "mlp_bf16", "mlp_f32"])
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--every", type=int, default=1000)
    ap.add_argument("--tau", type=float, default=0.51)
    ap.add_argument("--weights", default=None, help="torch.save'd packed weights (MLP kinds)")
    args = ap.parse_args()
    theta = None
    if args.weights:
        theta = inputs.load_weights(args.weights, "cuda")
    if args.compare:
        rec = long_comparison(theta, n=args.n, steps=args.steps, every=args.every, tau=args.tau)
        print(json.dumps({k: {f: v[f] for f in ("unstable_at", "mlups", "wall_s", "ess")}
                          | {"records": len(v["steps"]),
                             "energy_last": v["energy"][-1] if v["energy"] else None}
                          for k, v in rec.items()}))
        if args.out:
            with open(args.out, "w") as fh:
                json.dump(rec, fh)
        return
    res = run(n=args.n, kind=args.kind, steps=args.steps, every=args.every, tau=args.tau,
              theta=theta)
    S_mean = res["S"].mean(0)
    print(json.dumps({"kind": args.kind, "n": args.n, "steps": args.steps,
                      "mlups": round(res["mlups"], 1), "status": res["status"],
                      "energy": float(res["E"][-1].sum()),
                      "ess": [round(float(v), 4) for v in ess_exponents(S_mean)]}))


if __name__ == "__main__":
    main()

"""Benchmark of the D2Q9 learned-collision step (the hot path) on GB300.

Workload (one "step"): one fused pull-stream + learned-collision lattice-
Boltzmann step (MLP 9-64-64-9, tanh, BF16 tensor cores, FP32 populations,
Kolmogorov forcing by EDM) on a periodic 4096 x 4096 grid, the headline
configuration.  The state (2 x 604 MB) is larger than L2, so no flush is
needed between steps.  Also measured in the same run and reported under
"components": the plain BGK and Smagorinsky-BGK steps and the FP32 learned
step at 4096^2, and the unrolled training step (32 x 256^2 trajectories,
16 steps, checkpoint every 4) forward and forward+adjoint.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
N > 1 runs one independent replica per rank (launched by torch.distributed.run;
the path has no data exchange): weak scaling, value = sum over ranks.
--impl reference times the FP64 CPU oracle on this machine's host cores on a
bounded sample of the same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_GRID = 4096
TAU = 0.6
FORCE_AMP, FORCE_MODE = 1e-5, 4
METRIC = "MLUPS & %HBM/tensor roofline, D2Q9 learned-collision vs BGK at 4096²; fwd+adj ms/step"
BYTES_PER_NODE = 72  # algorithmic HBM traffic of one FP32 D2Q9 step: 36 B read + 36 B written
MLP_FLOP_PER_NODE = 2 * (9 * 64 + 64 * 64 + 64 * 9)  # 10,496 algorithmic flops of the MLP
# Xavier weights with the output layer scaled by 0.3: plain Xavier weights make
# the learned collision blow up within ~100 steps; 0.3 stays stable for >1500.
OUT_SCALE = 0.3
MLP_BF16_SOURCES = ("mlp_bf16.cu", "lattice.cuh", "umma.cuh", "kernels.h")
# Sub-partition cycles one warp-wide cvt.rn.bf16x2.f32 + tanh.approx.bf16x2 pair
# holds the XU (measured, profiles/activation_units_microbenchmark.md).
XU_PAIR_CYCLES = 16.42
WORKLOAD = ("D2Q9 learned-collision LBM step (MLP 9-64-64-9 tanh on tcgen05 BF16, FP32 "
            "populations), periodic 4096x4096, Kolmogorov forcing F0=1e-5 m=4, tau=0.6, "
            "random-phase initial field (rms 0.02, seed 2), Xavier weights (seed 3, output "
            "layer x0.3)")


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), float(p["bf16_tflops"]), "measured"
    except Exception:
        return 6800.0, 1900.0, "fallback"


class NvmlSampler:
    """Clock, throttle-reason and power sampling through NVML (read-only queries,
    ctypes) from a host thread every ~1 ms, so that a timed region of a few
    milliseconds still has samples inside it.  `mark(t0, t1)` records the host
    times of the timed region; only samples inside it are summarised."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, gpu_id=None, index=0):
        import ctypes as C
        import threading
        self.C = C
        lib = C.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        self.lib = lib
        self.h = C.c_void_p()
        # by UUID when known (NVML numbers the physical GPUs, whatever
        # CUDA_VISIBLE_DEVICES says), else by index
        rc = lib.nvmlDeviceGetHandleByUUID(C.c_char_p(gpu_id.encode()), C.byref(self.h)) \
            if gpu_id else lib.nvmlDeviceGetHandleByIndex_v2(C.c_uint(index), C.byref(self.h))
        if rc != 0:
            raise RuntimeError("no NVML handle")
        self.reason_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        self.rows, self.window = [], None
        self.stop = threading.Event()
        self.thread = threading.Thread(target=self._run, daemon=True)

    def _query(self):
        C, lib = self.C, self.lib
        clk, mx, pw, rs = C.c_uint(), C.c_uint(), C.c_uint(), C.c_ulonglong()
        lib.nvmlDeviceGetClockInfo(self.h, 1, C.byref(clk))      # NVML_CLOCK_SM
        lib.nvmlDeviceGetMaxClockInfo(self.h, 1, C.byref(mx))
        lib.nvmlDeviceGetPowerUsage(self.h, C.byref(pw))         # mW
        self.reason_fn(self.h, C.byref(rs))
        return clk.value, mx.value, pw.value / 1000.0, rs.value

    def _run(self):
        while not self.stop.is_set():
            self.rows.append((time.perf_counter(), *self._query()))
            time.sleep(0.001)

    def __enter__(self):
        self.thread.start()
        time.sleep(0.05)
        return self

    def __exit__(self, *a):
        self.stop.set()
        self.thread.join(timeout=5)

    def mark(self, t0, t1):
        self.window = (t0, t1)

    def summary(self):
        rows = self.rows
        if self.window:
            t0, t1 = self.window
            inside = [r for r in rows if t0 <= r[0] <= t1]
            rows = inside or rows
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        reasons = sorted({name for r in rows for bit, name in self.REASONS.items() if r[4] & bit})
        return {"sm_mhz": statistics.median(r[1] for r in rows), "sm_max_mhz": float(rows[0][2]),
                "reasons": reasons, "samples": len(rows), "power_w_max": max(r[3] for r in rows),
                "source": "nvml, ~1 ms, samples inside the timed region"}


def clock_sampler(gpu_id, index):
    """NVML sampling if the library loads, else nvidia-smi."""
    try:
        return NvmlSampler(gpu_id, index)
    except Exception:
        return ClockSampler(gpu_id)


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region (fallback)."""

    def mark(self, t0, t1):
        pass

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id=None):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def __enter__(self):
        import tempfile
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "100", "-f", self.path]
        if self.gpu_id:
            cmd[1:1] = ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
            os.unlink(self.path)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]),
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())
                if any(r[3].replace(".", "").isdigit() for r in rows) else None}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _init_pg(world, backend):
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist


def _max_over_ranks(x, world, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _initial_state(lbm, torch, dev, n=N_GRID, seed=2):
    from paper_2403_18466_gb300 import inputs
    rho, ux, uy = inputs.random_velocity_field(n, n, seed=seed, k0=8.0, urms=0.02)
    lat = lbm.Lattice(n, n, 1, tau=TAU, smag_cs=0.1, force_amp=FORCE_AMP, force_mode=FORCE_MODE,
                      device=dev)
    t = lambda a: torch.tensor(a[None], dtype=torch.float32, device=dev)
    lat.init_equilibrium(t(rho), t(ux), t(uy))
    return lat


def _time_steps(lat, kind, w, steps, torch, stream):
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    lat.step(steps, kind, w)
    end.record(stream)
    end.synchronize()
    return start.elapsed_time(end)  # ms


def _time_diagnostics(lat, n, torch, stream, hbm_peak):
    """On-device turbulence diagnostics of the n^2 state (the paper's
    evaluation quantities): the energy spectrum (velocity from the moments, one
    batched cuFFT R2C of both components, shell binning) and the longitudinal
    structure functions S^p(r), p = 1..6, r = 1..256 (u read once per
    separation: 8 B per node per r of algorithmic traffic)."""
    kmax, rmax = n // 2, 256
    out = {}
    for name, fn in (("energy_spectrum", lambda: lat.energy_spectrum(kmax)),
                     ("structure_functions_r256", lambda: lat.structure_functions(rmax))):
        fn()
        torch.cuda.synchronize()
        reps = 5
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        b.synchronize()
        out[name] = {"ms": round(a.elapsed_time(b) / reps, 3)}
    sf = out["structure_functions_r256"]
    g = 8.0 * n * n * rmax / (sf["ms"] * 1e-3) / 1e9
    sf["gbs"] = round(g, 1)
    sf["hbm_frac"] = round(g / hbm_peak, 4)
    out["grid"] = f"{n}x{n}"
    return out


def _time_steps_segments(lat, kind, w, steps, torch, stream, nseg=5):
    """The same timed region as _time_steps, issued as nseg back-to-back
    segments with an event between them (events do not stall the stream).
    Returns the whole region's ms and the per-step ms of each segment."""
    nseg = max(1, min(nseg, steps))
    sizes = [steps // nseg + (1 if i < steps % nseg else 0) for i in range(nseg)]
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(nseg + 1)]
    ev[0].record(stream)
    for i, k in enumerate(sizes):
        lat.step(k, kind, w)
        ev[i + 1].record(stream)
    ev[-1].synchronize()
    per_step = [ev[i].elapsed_time(ev[i + 1]) / k for i, k in enumerate(sizes)]
    return ev[0].elapsed_time(ev[-1]), per_step


def run_gpu(args):
    import torch
    from paper_2403_18466_gb300 import inputs, lbm

    world, rank, local = _dist()
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    _init_pg(world, "nccl")
    lbm.load()
    hbm_peak, tc_peak, peak_kind = _peaks()
    stream = torch.cuda.current_stream(dev)
    nodes = N_GRID * N_GRID

    lat = _initial_state(lbm, torch, dev)
    theta = torch.tensor(inputs.xavier_mlp(3, out_scale=OUT_SCALE), dtype=torch.float32,
                         device=dev)
    w = lbm.weights_struct(theta)

    # ---- headline: BF16 learned-collision steps -------------------------
    lat.step(max(3, args.warmup), "mlp_bf16", w)
    torch.cuda.synchronize()
    props = torch.cuda.get_device_properties(dev)
    uuid = getattr(props, "uuid", None)
    gpu_id = f"GPU-{uuid}" if uuid is not None and not str(uuid).startswith("GPU-") else (
        str(uuid) if uuid is not None else None)
    _barrier(world)
    torch.cuda.synchronize()
    with clock_sampler(gpu_id, local) as clk:
        t_host0 = time.perf_counter()
        ms, seg = _time_steps_segments(lat, "mlp_bf16", w, args.steps, torch, stream)
        clk.mark(t_host0, time.perf_counter())
    torch.cuda.synchronize()
    _barrier(world)
    ms_max = _max_over_ranks(ms, world, dev)
    status = lat.status()
    ms_step = ms_max / args.steps
    value = world * nodes / (ms_step * 1e-3) / 1e6  # MLUPS, whole job
    clocks = clk.summary()

    # ---- roofline of the dominant kernel (the step kernel itself) ---------
    achieved_gbs = BYTES_PER_NODE * nodes / (ms / args.steps * 1e-3) / 1e9
    # binding unit of the learned step: the XU (special-function) pipe.  Of
    # every 8 pairs of hidden units the compiled kernel sends `xu8` to the XU
    # (cvt.rn.bf16x2.f32 + tanh.approx.bf16x2) and the rest to the FMA pipe.
    # Measured on this GPU (profiles/activation_units_microbenchmark.md): one
    # warp-wide XU pair holds an SM sub-partition's XU for 16.42 cycles.  A node
    # has 64 pairs, so the XU needs 64 * xu8/8 * 16.42 / 32 sub-partition cycles
    # per node, a quarter of that in SM cycles.
    wg_per_sm, xu8 = lbm.mlp_bf16_layout()
    xu_sm_cycles_per_node = 64 * (xu8 / 8.0) * XU_PAIR_CYCLES / 32 / 4
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    node_rate = nodes / (ms / args.steps * 1e-3) / 1e6  # MLUPS per GPU
    xu_bound = sms * sm_mhz * 1e6 / xu_sm_cycles_per_node / 1e6 if xu8 else float("inf")
    binding = {"unit": "xu (tanh.approx.bf16x2 + cvt.rn.bf16x2.f32 of the XU pairs)",
               "achieved": round(node_rate, 1), "peak": round(xu_bound, 1), "peak_unit": "MLUPS",
               "frac": round(node_rate / xu_bound, 4),
               "sm_cycles_per_node": round(sms * sm_mhz * 1e6 / (node_rate * 1e6), 3),
               "xu_sm_cycles_per_node": round(xu_sm_cycles_per_node, 3),
               "time_x_sm_mhz": round(ms / args.steps * sm_mhz, 2),
               "kernel_layout": {"warpgroups_per_sm": wg_per_sm, "xu_pairs_of_8": xu8},
               "derivation": f"64 hidden-unit pairs per node, {xu8} of 8 on the XU at "
                             f"{XU_PAIR_CYCLES} sub-partition cycles per warp-wide pair "
                             "(measured), 4 sub-partitions per SM, measured SM clock"}
    # the other bound next to the XU: instruction issue (ALU, FMA, XU, memory
    # and tensor-memory instructions all take issue slots)
    issue = _issue_bound(MLP_BF16_SOURCES, "k_step_mlp_bf16_2048.md", sms, sm_mhz)
    if issue:
        issue["frac"] = round(node_rate / issue["peak"], 4)
    binding["issue"] = issue
    roofline = {"bound": "hbm", "achieved": round(achieved_gbs, 1), "peak": hbm_peak,
                "unit": "GB/s", "frac": round(achieved_gbs / hbm_peak, 4),
                "traffic": _traffic_from_profile(MLP_BF16_SOURCES, "k_step_mlp_bf16_2048.md", nodes),
                "peak_source": peak_kind,
                "kernel": "k_step_mlp_bf16",
                "tensor_frac": round(MLP_FLOP_PER_NODE * nodes / (ms / args.steps * 1e-3)
                                     / (tc_peak * 1e12), 4)}

    # ---- components, same run ------------------------------------------------
    comps = {}
    for kind, k in (("bgk", max(args.steps, 200)), ("smag", max(args.steps, 200)),
                    ("mlp_f32", max(5, args.steps // 50))):
        lat.step(3, kind, w)
        t = _time_steps(lat, kind, w, k, torch, stream)
        g = BYTES_PER_NODE * nodes / (t / k * 1e-3) / 1e9
        comps[kind] = {"mlups": round(nodes / (t / k * 1e-3) / 1e6, 1),
                       "ms_per_step": round(t / k, 5), "hbm_gbs": round(g, 1),
                       "hbm_frac": round(g / hbm_peak, 4)}
    comps["mlp_bf16"] = {"mlups": round(nodes / (ms_step * 1e-3) / 1e6, 1),
                         "ms_per_step": round(ms_step, 5), "hbm_gbs": roofline["achieved"],
                         "hbm_frac": roofline["frac"], "weights": "xavier seed 3, output x0.3"}
    # the same step with the trained weights (the configuration names seeded
    # Xavier weights and trained weights), from the same initial state
    wt = lbm.weights_struct(inputs.trained_mlp(dev))
    lat_t = _initial_state(lbm, torch, dev)
    lat_t.step(3, "mlp_bf16", wt)
    kt = max(50, args.steps // 10)
    t = _time_steps(lat_t, "mlp_bf16", wt, kt, torch, stream)
    g = BYTES_PER_NODE * nodes / (t / kt * 1e-3) / 1e9
    comps["mlp_bf16_trained"] = {"mlups": round(nodes / (t / kt * 1e-3) / 1e6, 1),
                                 "ms_per_step": round(t / kt, 5), "hbm_gbs": round(g, 1),
                                 "hbm_frac": round(g / hbm_peak, 4), "steps": kt,
                                 "weights": "trained (paper_2403_18466_gb300/weights)",
                                 "status": lbm.lbm_strerror(lat_t.status())}
    del lat_t
    comps["training"] = _time_training(lbm, torch, dev, inputs)
    comps["diagnostics"] = _time_diagnostics(lat, N_GRID, torch, stream, hbm_peak)
    comps["d3q19"] = _time_d3q19(lbm, torch, dev, inputs, hbm_peak)
    del lat
    torch.cuda.empty_cache()

    # ---- end to end through the C ABI with host buffers ----------------------
    e2e = _time_e2e(lbm, torch, dev, inputs, w, args.steps, world)

    line = {
        "metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": round(ms_step, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "nx": N_GRID, "ny": N_GRID, "batch": 1,
                   "mlp_dtype": "bf16 (tcgen05, fp32 accumulate)", "population_dtype": "f32",
                   "l2": "inputs larger than L2 (state 2 x 604 MB), no flush",
                   "parallelism": f"replicas{world}"},
        "roofline": roofline, "binding_unit": binding, "clocks": clocks, "e2e": e2e,
        "gpu_launches": args.steps, "components": comps, "status": lbm.lbm_strerror(status),
        "segments": {"n": len(seg), "ms_per_step_median": round(statistics.median(seg), 5),
                     "ms_per_step_best": round(min(seg), 5),
                     "ms_per_step_worst": round(max(seg), 5)},
    }
    if rank == 0:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _time_training(lbm, torch, dev, inputs):
    """Unrolled training step: 32 x 256^2 trajectories, 16 LES steps, checkpoint
    every 4; forward (learned collision with checkpoints) and forward + velocity
    loss + hand-written adjoint, for the FP32 pair (CUDA-core MLP and adjoint)
    and the BF16 pair (tensor-core MLP and tensor-core adjoint)."""
    B, n, L, ck = 32, 256, 16, 4
    lat = lbm.Lattice(n, n, B, tau=0.500375, force_amp=8e-5, force_mode=4, device=dev)
    rho = torch.ones((B, n, n), device=dev)
    ux = torch.tensor(inputs.noise((B, n, n), 5, 0.02), dtype=torch.float32, device=dev)
    uy = torch.tensor(inputs.noise((B, n, n), 6, 0.02), dtype=torch.float32, device=dev)
    lat.init_equilibrium(rho, ux, uy)
    f0 = lat.get_state()
    theta = torch.tensor(inputs.xavier_mlp(3, out_scale=0.01), dtype=torch.float32, device=dev)
    w = lbm.weights_struct(theta)
    ws = torch.empty(lat.record_bytes(L, ck) // 4, dtype=torch.float32, device=dev)
    dW = torch.empty(lbm.LBM_MLP_NPARAMS, dtype=torch.float32, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    nodes = B * n * n
    out = {"config": "32 x 256^2, 16 steps, checkpoint every 4"}
    for prec in ("f32", "bf16"):
        res = {}
        for rep in range(3):
            # the same 16 steps without a record (the inference forward)
            lat.set_state(f0)
            ev[0].record()
            lat.step(L, "mlp_f32" if prec == "f32" else "mlp_bf16", w)
            ev[1].record()
            ev[1].synchronize()
            plain_ms = ev[0].elapsed_time(ev[1])
            lat.set_state(f0)
            ev[0].record()
            lat.forward_record(L, ck, w, ws, prec)
            ev[1].record()
            loss, g = lat.velocity_loss(ux, uy)
            lat.backward(g, w, ws, dW, None, prec)
            ev[2].record()
            ev[2].synchronize()
            res = {"fwd_ms": ev[0].elapsed_time(ev[1]), "fwd_adj_ms": ev[0].elapsed_time(ev[2]),
                   "plain_ms": plain_ms}
        out[prec] = {"fwd_ms_per_step": round(res["fwd_ms"] / L, 4),
                     "fwd_adj_ms_per_step": round(res["fwd_adj_ms"] / L, 4),
                     "ratio_fwd_adj_over_fwd": round(res["fwd_adj_ms"] / res["fwd_ms"], 3),
                     "fwd_mlups": round(nodes * L / (res["fwd_ms"] * 1e-3) / 1e6, 1),
                     "plain_fwd_ms_per_step": round(res["plain_ms"] / L, 4),
                     "ratio_fwd_adj_over_plain_fwd": round(res["fwd_adj_ms"] / res["plain_ms"], 3)}
    out["ratio_bf16_fwd_adj_over_f32_fwd"] = round(
        out["bf16"]["fwd_adj_ms_per_step"] / out["f32"]["fwd_ms_per_step"], 3)
    # the memory / recompute trade of the checkpoint interval k (tensor-core
    # pair, same 16-step unroll): the backward recomputes the k - 1 inner
    # states of every segment but the last (which the record keeps) and the
    # workspace holds ceil(16/k) + k + 1 states
    sweep = {}
    for ck_i in (1, 2, 4, 8, 16):
        ws_i = torch.empty(lat.record_bytes(L, ck_i) // 4, dtype=torch.float32, device=dev)
        for rep in range(3):
            lat.set_state(f0)
            ev[0].record()
            lat.forward_record(L, ck_i, w, ws_i, "bf16")
            ev[1].record()
            loss, g = lat.velocity_loss(ux, uy)
            lat.backward(g, w, ws_i, dW, None, "bf16")
            ev[2].record()
            ev[2].synchronize()
            res = {"fwd_ms": ev[0].elapsed_time(ev[1]), "fwd_adj_ms": ev[0].elapsed_time(ev[2])}
        sweep[str(ck_i)] = {"fwd_ms_per_step": round(res["fwd_ms"] / L, 4),
                            "fwd_adj_ms_per_step": round(res["fwd_adj_ms"] / L, 4),
                            "ratio_fwd_adj_over_fwd": round(res["fwd_adj_ms"] / res["fwd_ms"], 3),
                            "workspace_mb": round(ws_i.numel() * 4 / 2**20, 1)}
        del ws_i
    out["bf16_checkpoint_every"] = sweep
    # the paper's training variant: population loss (Eq. S13) on |S| = 512
    # random nodes after L_T = 12 or 24 unrolled steps, tensor-core pair
    gen = torch.Generator().manual_seed(11)
    idx = torch.randperm(nodes, generator=gen)[:512].to(device=dev, dtype=torch.int32)
    target = lat.stream(f0, -1)
    for LT in (12, 24):
        ws = torch.empty(lat.record_bytes(LT, ck) // 4, dtype=torch.float32, device=dev)
        for rep in range(3):
            lat.set_state(f0)
            ev[0].record()
            lat.forward_record(LT, ck, w, ws, "bf16")
            ev[1].record()
            loss, g = lat.population_loss_subset(idx, target)
            lat.backward(g, w, ws, dW, None, "bf16")
            ev[2].record()
            ev[2].synchronize()
            res = {"fwd_ms": ev[0].elapsed_time(ev[1]), "fwd_adj_ms": ev[0].elapsed_time(ev[2])}
        out[f"bf16_subset512_population_LT{LT}"] = {
            "fwd_adj_ms": round(res["fwd_adj_ms"], 3),
            "fwd_adj_ms_per_step": round(res["fwd_adj_ms"] / LT, 4),
            "ratio_fwd_adj_over_fwd": round(res["fwd_adj_ms"] / res["fwd_ms"], 3),
            "workspace_mb": round(ws.numel() * 4 / 2**20, 1)}
        del ws
    return out


def _time_d3q19(lbm, torch, dev, inputs, hbm_peak):
    """The paper's 3D setting: D3Q19 BGK and Smagorinsky steps at 256^3
    (152 B/node of algorithmic traffic) and the FP32 learned collision with the
    paper's 19-300-300-100-19 network at 64^3."""
    import numpy as np
    out = {}
    n = 256
    # a 64^3 solenoidal field tiled 4 x 4 x 4 (periodic, still solenoidal)
    rho, u = inputs.random_velocity_field_3d(64, 64, 64, seed=3, k0=4.0, urms=0.02)
    rho, u = np.tile(rho, (4, 4, 4)), np.tile(u, (1, 4, 4, 4))
    lat = lbm.Lattice3D(n, n, n, 1, tau=0.51, smag_cs=0.1, force_amp=1e-6, device=dev)
    lat.init_equilibrium(torch.tensor(rho[None], dtype=torch.float32, device=dev),
                         torch.tensor(u[None], dtype=torch.float32, device=dev))
    del rho, u
    stream = torch.cuda.current_stream(dev)
    nodes = n ** 3
    for kind, k in (("bgk", 50), ("smag", 50)):
        lat.step(3, kind)
        t = _time_steps(lat, kind, None, k, torch, stream)
        g = 152 * nodes / (t / k * 1e-3) / 1e9
        out[f"{kind}_256^3"] = {"mlups": round(nodes / (t / k * 1e-3) / 1e6, 1),
                                "ms_per_step": round(t / k, 4), "hbm_gbs": round(g, 1),
                                "hbm_frac": round(g / hbm_peak, 4)}
    out["status"] = lbm.lbm_strerror(lat.status())
    del lat
    torch.cuda.empty_cache()
    n = 64
    rho, u = inputs.random_velocity_field_3d(n, n, n, seed=4, k0=4.0, urms=0.02)
    lat = lbm.Lattice3D(n, n, n, 1, tau=0.6, device=dev)
    lat.init_equilibrium(torch.tensor(rho[None], dtype=torch.float32, device=dev),
                         torch.tensor(u[None], dtype=torch.float32, device=dev))
    theta = torch.tensor(inputs.xavier_mlp_widths(5, (300, 300, 100), out_scale=0.01),
                         dtype=torch.float32, device=dev)
    w3 = lbm.weights3d_struct(theta)
    lat.step(1, "mlp_f32", w3)
    k = 5
    t = _time_steps(lat, "mlp_f32", w3, k, torch, stream)
    flop = 2 * (19 * 300 + 300 * 300 + 300 * 100 + 100 * 19)
    out["mlp_f32_64^3"] = {"mlups": round(n ** 3 / (t / k * 1e-3) / 1e6, 1),
                           "ms_per_step": round(t / k, 3),
                           "mlp_tflops": round(flop * n ** 3 / (t / k * 1e-3) / 1e12, 2),
                           "status": lbm.lbm_strerror(lat.status())}
    del lat
    torch.cuda.empty_cache()
    # tensor-core collision at 256^3 (the 64^3 field tiled, as above)
    n = 256
    rho, u = inputs.random_velocity_field_3d(64, 64, 64, seed=4, k0=4.0, urms=0.02)
    rho, u = np.tile(rho, (4, 4, 4)), np.tile(u, (1, 4, 4, 4))
    lat = lbm.Lattice3D(n, n, n, 1, tau=0.6, force_amp=1e-6, device=dev)
    lat.init_equilibrium(torch.tensor(rho[None], dtype=torch.float32, device=dev),
                         torch.tensor(u[None], dtype=torch.float32, device=dev))
    del rho, u
    lat.step(3, "mlp_bf16", w3)
    k = 20
    t = _time_steps(lat, "mlp_bf16", w3, k, torch, stream)
    rate = n ** 3 / (t / k * 1e-3)
    _, tc_peak, _ = _peaks()
    out["mlp_bf16_256^3"] = {"mlups": round(rate / 1e6, 1), "ms_per_step": round(t / k, 4),
                             "mlp_tflops": round(flop * rate / 1e12, 1),
                             "tensor_frac": round(flop * rate / 1e12 / tc_peak, 4),
                             "flop_per_node": flop,
                             "status": lbm.lbm_strerror(lat.status())}
    return out


def _time_e2e(lbm, torch, dev, inputs, w, steps, world):
    """The same workload through lbm_run_host: pinned host populations in,
    `steps` learned-collision steps, density and velocity back to pinned host
    memory, all inside the timed region (host clock around a synchronous call)."""
    n = N_GRID
    rho, ux, uy = inputs.random_velocity_field(n, n, seed=2, k0=8.0, urms=0.02)
    lat = _initial_state(lbm, torch, dev)
    f_host = lat.get_state().cpu().pin_memory()
    outs = [torch.empty((1, n, n), dtype=torch.float32).pin_memory() for _ in range(3)]
    lat.run_host(f_host, 3, "mlp_bf16", w, *outs)  # warm-up
    _barrier(world)
    t0 = time.perf_counter()
    lat.run_host(f_host, steps, "mlp_bf16", w, *outs)
    dt = time.perf_counter() - t0
    dt = _max_over_ranks(dt, world, dev)
    h2d = f_host.numel() * 4
    d2h = 3 * n * n * 4
    return {"value": round(world * n * n * steps / dt / 1e6, 1), "unit": "MLUPS",
            "h2d_bytes_per_step": h2d / steps, "d2h_bytes_per_step": d2h / steps,
            "note": f"lbm_run_host: {h2d} B in, {steps} steps, {d2h} B out per call"}


def cpu_baseline(seconds=12.0, n=1024):
    """The FP64 oracle (as it stands) on this machine's host cores: learned
    collision steps on an n x n crop of the same recipe, as many steps as fit
    in about `seconds`."""
    import numpy as np

    import oracle
    from paper_2403_18466_gb300 import inputs
    rho, ux, uy = inputs.random_velocity_field(n, n, seed=2, k0=8.0 * n / N_GRID, urms=0.02)
    g = oracle.stream_push(oracle.equilibrium_field(rho[None], ux[None], uy[None]))
    prm = oracle.params(TAU, force_amp=FORCE_AMP, force_mode=FORCE_MODE)
    theta = inputs.xavier_mlp(3, out_scale=OUT_SCALE)
    t0 = time.perf_counter()
    g = oracle.step(oracle.MLP, g, prm, theta)
    one = time.perf_counter() - t0
    k = max(1, min(50, int(seconds / max(one, 1e-6))))
    t0 = time.perf_counter()
    oracle.run(oracle.MLP, g, k, prm, theta)
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    out = {"value": round(n * n * k / dt / 1e6, 3), "unit": "MLUPS", "cores": cores,
           "kind": "oracle",
           "sample": f"FP64 oracle, learned collision, {n}x{n} crop of the same recipe, "
                     f"{k} steps, {dt:.1f} s"}
    # the other collisions on all cores, and the learned one on a single core
    # (a child process, so that its OpenMP runtime starts with one thread)
    comps = {}
    for name, kind in (("bgk", oracle.BGK), ("smag", oracle.SMAG)):
        prm_k = oracle.params(TAU, smag_cs=0.1 if kind == oracle.SMAG else 0.0,
                              force_amp=FORCE_AMP, force_mode=FORCE_MODE)
        t0 = time.perf_counter()
        oracle.run(kind, g, 20, prm_k)
        t = time.perf_counter() - t0
        comps[f"{name}_{n}^2_20_steps"] = {"mlups": round(n * n * 20 / t / 1e6, 3),
                                           "cores": cores}
    code = ("import time, oracle; from paper_2403_18466_gb300 import inputs; import bench;"
            "r, u, v = inputs.random_velocity_field(256, 256, seed=2, k0=0.5, urms=0.02);"
            "g = oracle.stream_push(oracle.equilibrium_field(r[None], u[None], v[None]));"
            "p = oracle.params(bench.TAU, force_amp=bench.FORCE_AMP, force_mode=bench.FORCE_MODE);"
            "th = inputs.xavier_mlp(3, out_scale=bench.OUT_SCALE);"
            "t0 = time.perf_counter(); oracle.run(oracle.MLP, g, 5, p, th);"
            "print(256 * 256 * 5 / (time.perf_counter() - t0) / 1e6)")
    try:
        env = dict(os.environ, OMP_NUM_THREADS="1")
        res = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env,
                             capture_output=True, text=True, timeout=120)
        comps["mlp_256^2_5_steps_1_core"] = {"mlups": round(float(res.stdout.strip().splitlines()[-1]), 3),
                                             "cores": 1}
    except Exception as e:  # the single-core figure is informative only
        comps["mlp_256^2_5_steps_1_core"] = {"unavailable": str(e)[:200]}
    out["components"] = comps
    return out


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return
    import numpy as np

    import oracle
    from paper_2403_18466_gb300 import inputs
    prm = oracle.params(TAU, force_amp=FORCE_AMP, force_mode=FORCE_MODE)
    theta = inputs.xavier_mlp(3, out_scale=OUT_SCALE)
    # each step is one oracle step on an n x n crop of the same recipe; the crop
    # is the largest of 512, 256, 128, 64 for which all K steps fit ~90 s
    budget = 90.0
    for n in (512, 256, 128, 64):
        rho, ux, uy = inputs.random_velocity_field(n, n, seed=2, k0=max(1.0, 8.0 * n / N_GRID),
                                                   urms=0.02)
        g = oracle.stream_push(oracle.equilibrium_field(rho[None], ux[None], uy[None]))
        t0 = time.perf_counter()
        g = oracle.step(oracle.MLP, g, prm, theta)  # warm-up and estimate
        one = time.perf_counter() - t0
        if one * args.steps <= budget:
            break
    for _ in range(max(0, args.warmup - 1)):
        if one * (args.warmup + args.steps) > 2 * budget:
            break
        g = oracle.step(oracle.MLP, g, prm, theta)
    k = args.steps
    t0 = time.perf_counter()
    for _ in range(k):
        g = oracle.step(oracle.MLP, g, prm, theta)
    dt = time.perf_counter() - t0
    value = n * n * k / dt / 1e6
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = f"FP64 oracle, learned collision, {n}x{n} crop of the 4096^2 recipe, {k} steps"
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "MLUPS",
            "n_gpus": world, "steps": k, "warmup": args.warmup, "ms_per_step": round(dt / k * 1e3, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "nx": N_GRID, "ny": N_GRID, "batch": 1,
                       "sample": sample},
            "cpu_baseline": {"value": round(value, 3), "unit": "MLUPS", "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_profile_case(args):
    """Small case for ncu: `--steps` steps of one collision kind on a
    `--grid` x `--grid` lattice, or one training step (`adjoint_bf16`); no JSON
    line."""
    import torch
    from paper_2403_18466_gb300 import inputs, lbm
    dev = torch.device("cuda:0")
    lbm.load()
    if args.profile.startswith("d3_"):
        # D3Q19 (the paper's 3D setting) on a --grid^3 lattice
        kind, n = args.profile[3:], args.grid
        rho, u = inputs.random_velocity_field_3d(n, n, n, seed=4, k0=4.0, urms=0.02)
        lat = lbm.Lattice3D(n, n, n, 1, tau=0.6, force_amp=1e-6, device=dev)
        lat.init_equilibrium(torch.tensor(rho[None], dtype=torch.float32, device=dev),
                             torch.tensor(u[None], dtype=torch.float32, device=dev))
        theta = torch.tensor(inputs.xavier_mlp_widths(5, (300, 300, 100), out_scale=0.01),
                             dtype=torch.float32, device=dev)
        lat.step(args.steps, kind, lbm.weights3d_struct(theta))
        torch.cuda.synchronize()
        rc = lat.status()
        print(f"profile case {args.profile} {n}^3 x {args.steps}: {lbm.lbm_strerror(rc)}")
        if rc != lbm.LBM_OK:
            sys.exit(1)
        return
    if args.profile in ("adjoint_bf16", "adjoint_f32"):
        # one unrolled training step of the tensor-core (or FP32) pair: 32
        # trajectories of --grid^2, --steps LES steps, checkpoint every 4
        prec = args.profile.split("_")[1]
        B, n, L = 32, args.grid, args.steps
        lat = lbm.Lattice(n, n, B, tau=0.500375, force_amp=8e-5, force_mode=4, device=dev)
        ux = torch.tensor(inputs.noise((B, n, n), 5, 0.02), dtype=torch.float32, device=dev)
        uy = torch.tensor(inputs.noise((B, n, n), 6, 0.02), dtype=torch.float32, device=dev)
        lat.init_equilibrium(torch.ones((B, n, n), device=dev), ux, uy)
        theta = torch.tensor(inputs.xavier_mlp(3, out_scale=0.01), dtype=torch.float32,
                             device=dev)
        w = lbm.weights_struct(theta)
        ws = torch.empty(lat.record_bytes(L, 4) // 4, dtype=torch.float32, device=dev)
        dW = torch.empty(lbm.LBM_MLP_NPARAMS, dtype=torch.float32, device=dev)
        lat.forward_record(L, 4, w, ws, prec)
        _, g = lat.velocity_loss(ux, uy)
        lat.backward(g, w, ws, dW, None, prec)
        torch.cuda.synchronize()
        rc = lat.status()
        print(f"profile case {args.profile} 32 x {n}^2 x {L}: {lbm.lbm_strerror(rc)}")
        if rc != lbm.LBM_OK:
            sys.exit(1)
        return
    lat = _initial_state(lbm, torch, dev, n=args.grid)
    theta = torch.tensor(inputs.xavier_mlp(3, out_scale=OUT_SCALE), dtype=torch.float32,
                         device=dev)
    w = lbm.weights_struct(theta)
    lat.step(args.steps, args.profile, w)
    torch.cuda.synchronize()
    rc = lat.status()
    print(f"profile case {args.profile} {args.grid}^2 x {args.steps}: {lbm.lbm_strerror(rc)}")
    if rc != lbm.LBM_OK:
        sys.exit(1)


def kernel_code_digest(kernel_sources):
    """SHA-256 of the kernel sources with // comments and blank lines removed,
    so that a comment edit does not void a capture but any code change does."""
    import hashlib
    h = hashlib.sha256()
    for src in kernel_sources:
        with open(os.path.join(ROOT, "paper_2403_18466_gb300", "csrc", src)) as fh:
            for line in fh:
                code = line.split("//", 1)[0].rstrip() if '"' not in line else line.rstrip()
                if code.strip():
                    h.update((code + "\n").encode())
    return h.hexdigest()


def _profile_fields(kernel_sources, summary):
    """The "- key: value" fields of a committed ncu summary, or None if the
    kernel code changed since the capture (or the summary is unreadable)."""
    path = os.path.join(ROOT, "profiles", summary)
    try:
        fields = {}
        for line in open(path):
            if ":" in line and line.strip().startswith("- "):
                k, v = line.strip()[2:].split(":", 1)
                fields[k.strip()] = v.strip().strip("`")
        if fields.get("code_sha256") != kernel_code_digest(kernel_sources):
            return None
        return fields
    except Exception:
        return None


def _traffic_from_profile(kernel_sources, summary, nodes):
    """DRAM bytes per launch of the step kernel from a committed ncu summary,
    scaled to `nodes`; None if the kernel code changed since the capture."""
    f = _profile_fields(kernel_sources, summary)
    try:
        return float(f["dram_bytes_per_launch"]) * nodes / float(f["nodes_per_launch"])
    except Exception:
        return None


def _issue_bound(kernel_sources, summary, sms, sm_mhz):
    """Instruction-issue bound of the step kernel: its warp instructions per
    node (committed ncu summary; None once the kernel code has changed) at four
    warp instructions per SM cycle (one per sub-partition), in MLUPS."""
    f = _profile_fields(kernel_sources, summary)
    try:
        per_node = float(f["warp_instructions_per_launch"]) / float(f["nodes_per_launch"])
    except Exception:
        return None
    cycles = per_node / 4.0
    return {"peak": round(sms * sm_mhz / cycles, 1), "peak_unit": "MLUPS",
            "warp_instructions_per_node": round(per_node, 2),
            "sm_cycles_per_node": round(cycles, 3),
            "source": f"profiles/{summary} (smsp__inst_executed.sum of one launch)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--profile", default=None,
                    choices=["bgk", "smag", "mlp_bf16", "mlp_f32", "d3_bgk", "d3_smag",
                             "d3_mlp_bf16", "d3_mlp_f32", "adjoint_bf16", "adjoint_f32"],
                    help="run a small case of one kernel for ncu and exit")
    ap.add_argument("--grid", type=int, default=2048)
    args = ap.parse_args()
    if args.profile:
        run_profile_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()

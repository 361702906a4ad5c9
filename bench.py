"""Benchmark: extended-model gradient throughput on the guided-wave workload.

Workload: 1000x300 grid (dx = 1 m), 30 m shale waveguide with +-3 % random
perturbations, 32 moment-tensor sources (one extended component each), 500
DAS channels (1 m spacing, 10 m gauge), nt = 4000 (dt = 0.1 ms), FP32 time
stepping.  One step = one extended-model gradient: data misfit and the
gradients of all 32 components (forward, checkpoint recompute, adjoint,
imaging, chain rule) plus the consistency-term gradient of Vp, Vs and rho.

Metric: G cell-updates/s, one cell-update = one physical cell x one time
step x one shot, counted once per gradient (ns * nx * nz * nt / seconds);
seconds per gradient are reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs its own copy of the workload (independent
extended problems, weak scaling); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gcell-updates/s and s per extended-model gradient (all shots) vs plain FP32 path"
UNIT = "Gcell-updates/s"
WORKLOAD = "guided_wave_1000x300: 32 shots x 500 DAS ch, nt=4000, dt=0.1ms, dx=1m, extended gradient + regularization"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--exec", default="batched", choices=["batched", "plain"])
    ap.add_argument("--ckpt-store", default="fp32", choices=["fp32", "fp16", "bf16"])
    ap.add_argument("--snap-store", default="fp32", choices=["fp32", "fp16", "bf16"],
                    help="precision of the stored forward velocities")
    ap.add_argument("--ckpt", default="auto",
                    help="checkpoint interval: 0 = sqrt(nt), n, or auto (every step stored when it fits, "
                         "else sqrt(nt) with as many final steps kept by the forward pass as fit)")
    ap.add_argument("--stored-steps", type=int, default=0,
                    help="final steps kept by the forward pass with an explicit interval")
    ap.add_argument("--no-sqrt", action="store_true",
                    help="skip the record of the sqrt(nt) schedule (no steps kept by the forward pass)")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP32 comparison run")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--stencil", default="auto", choices=["auto", "loads", "tma", "tma_pairs", "tma_staged"])
    ap.add_argument("--tile", default="0x0", help="forward tile, e.g. 32x16 (0x0 = autotune)")
    ap.add_argument("--adj-stencil", default="auto", choices=["auto", "loads", "tma"])
    ap.add_argument("--adj-tile", default="0x0", help="adjoint tile (0x0 = autotune)")
    ap.add_argument("--overlap", default="auto", choices=["auto", "off", "on"])
    ap.add_argument("--adj-form", default="auto", choices=["auto", "stress", "scaled"],
                    help="adjoint stress variable: sigma^ (stress) or F = dt C sigma^ (scaled)")
    ap.add_argument("--no-reduced", action="store_true", help="skip the reduced-storage record")
    ap.add_argument("--full-iteration-groups", type=int, default=1,
                    help="shot groups of the 4000x1200 full-iteration record to time (16 = all; 0 = skip)")
    ap.add_argument("--ns", type=int, default=32)
    ap.add_argument("--nt", type=int, default=4000)
    return ap.parse_args()


def rank_info():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def problem(ns, nt):
    import workloads as W
    p = W.guided_wave_1000x300(ns=ns, nt=nt)
    f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    p.acq.wavelet = f32(p.acq.wavelet)
    return p


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# Algorithmic bytes per padded cell of one launch of the two stencil kernels (what each
# launch must move at least once; FP32 words unless stated):
#   fused forward step: read vx vz sxx szz sxz + lambda mu mu_xz b_x b_z, write 5 = 60 B;
#     a launch that keeps v^{n+1/2} for the adjoint also writes vx, vz once more (8 B in FP32,
#     4 B as FP16/BF16 snapshots)
#   fused adjoint step: read 5 adjoint fields + 5 materials + 5 imaging sums, write 5 + 5
#     = 100 B, plus the forward vx, vz of the step (8 B FP32, 4 B FP16/BF16); the same in
#     the scaled-stress form, whose 5 adjoint fields hold v^ and F = dt C sigma^ and whose
#     materials (b_x, b_z on the velocity halo, lambda, mu, mu_xz on the tile) are read once
#   plain stress half-step: read vx vz + 3 stresses + lambda mu mu_xz, write 3 = 44 B
#   plain adjoint stress half-step: read 2 + 2 + 3 + 3 + 2 + 3, write 3 + 3 = 84 B
KERNELS = {
    ("batched", "step"): "forward_step (velocity + stress + source, all shots)",
    ("batched", "adj"): "adjoint_step (transposed step + imaging, all shots)",
    ("plain", "step"): "k_stress (forward stress half-step, one shot)",
    ("plain", "adj"): "k_adj_stress (adjoint stress half-step + imaging, one shot)",
}
NOMINAL_HBM_GBS = 7900.0


def snap_bytes(info):
    """Bytes of one stored forward-velocity element (FP32, or FP16/BF16 snapshots)."""
    return 4.0 if info.get("snap_store", 0) == 0 else 2.0


def recomputed_steps(info, nt):
    """Steps the adjoint recomputes from checkpoints: those before the first step the
    forward pass keeps (none with every step stored)."""
    return 0 if info["ckpt_interval"] >= nt else nt - info["stored_steps"]


def schedule_name(info, nt):
    if info["ckpt_interval"] >= nt:
        return "every step stored"
    if info["stored_steps"] == 0:
        return "sqrt(nt) checkpoints + recompute"
    return (f"sqrt(nt) checkpoints + recompute of the first {nt - info['stored_steps']} steps, "
            f"final {info['stored_steps']} kept by the forward pass")


def kernel_bytes(exec_, info, nt):
    """Algorithmic bytes per padded cell of the average forward-step launch of one
    gradient and of the adjoint-step launch.  Every step's v^{n+1/2} is written once,
    by the forward pass or by its recompute, so of the nt + (recomputed steps)
    forward-step launches nt write it."""
    if exec_ == "plain":
        return 44.0, 84.0
    v = 2 * snap_bytes(info)
    nrec = recomputed_steps(info, nt)
    return 60.0 + v * nt / (nt + nrec), 100.0 + v


# DRAM traffic per padded cell of one launch (dram__bytes_read.sum + dram__bytes_write.sum) from the ncu
# captures of the 8-shot case of this workload with the same kernel variant, scaled to a launch by its
# cells.  Keyed by (kernel, staging, tile, variant details, snapshot store); the forward step has one
# figure for a step that writes no velocities ("pass") and one for a step that keeps them ("keep"), mixed
# in the proportion of the gradient's schedule.  Any other variant, or a kernel changed since its
# capture, reports traffic null.
TRAFFIC_PER_CELL = {
    # forward step, TMA cell pairs, tile 32x16
    ("step", 3, 32, 16, 3, 0, 0): {"pass": 54.51, "keep": 59.79},
    # the same with FP16 snapshots (every step stored, per-thread stores)
    ("step", 3, 32, 16, 3, 0, 1): {"keep": 57.31},
    # adjoint step, scaled-stress form, TMA staging, cell pairs, tile 32x16, FP32 velocities / FP16 snapshots
    ("adj", 2, 32, 16, 2, 2, 0): 97.62,
    ("adj", 2, 32, 16, 3, 2, 0): 97.60,    # the same cell pairs in 512-thread CTAs
    ("adj", 2, 32, 16, 2, 2, 1): 92.78,
    # adjoint step (stress form), per-thread loads, tile 32x16, persistent grid, FP32 velocities
    ("adj", 1, 32, 16, 1, 1, 0): 94.97,
    # the stress-form adjoint with FP16 snapshots (every step stored)
    ("adj", 1, 32, 16, 1, 1, 1): 90.35,
}


# Algorithmic bytes of one whole gradient per padded cell and time step: the forward
# pass (60 B), the recompute of every checkpoint segment, which also keeps vx, vz of
# each step (60 + 8 B), and the adjoint step (100 + 8 B).  With every step stored the
# recompute drops and the forward pass keeps the velocities: 68 + 108 = 176 B, the floor
# of the method with FP32 velocities (forward, adjoint, velocity hand-off, imaging
# sums); FP16/BF16 snapshots halve the hand-off (168 B, or 228 B with the recompute).
# Steps kept by the forward pass are not recomputed: 176 + 60 x (recomputed / nt) B.
GRAD_FLOOR_BYTES = 176.0


def gradient_roofline(info, nt, s_per_grad):
    """Bandwidth of the whole gradient (one GPU's shots, every kernel of the step
    included) at the algorithmic bytes of its schedule and at the FP32 floor of 176 B
    per padded cell-step, both against the measured HBM peak."""
    hbm, peak_kind = peaks()
    v = 2 * snap_bytes(info)
    bpc = 60.0 + 60.0 * recomputed_steps(info, nt) / nt + (v + 100.0 + v)
    work = info["padded_cells"] * nt / s_per_grad / 1e9
    return {"bound": "hbm", "unit": "GB/s", "peak": hbm, "peak_kind": peak_kind,
            "schedule": schedule_name(info, nt),
            "snapshots": {0: "fp32", 1: "fp16", 2: "bf16"}[info.get("snap_store", 0)],
            "bytes_per_cell_step": bpc, "achieved": bpc * work, "frac": bpc * work / hbm,
            "floor_bytes_per_cell_step": GRAD_FLOOR_BYTES, "floor_frac": GRAD_FLOOR_BYTES * work / hbm}


def roofline(exec_, info, prof, nt, ns):
    """Roofline entries of the dominant and of the other stencil kernel: achieved =
    algorithmic bytes x cells of a launch / its mean CUDA-event duration, as a fraction
    of the measured HBM peak (frac) and of the nominal 7.9 TB/s (frac_nominal); with
    an ncu capture of the variant, the DRAM bytes it moved per launch (traffic) and
    traffic / duration as a fraction of the measured peak (frac_traffic)."""
    hbm, peak_kind = peaks()
    cells = info["padded_cells"] if exec_ == "batched" else info["padded_cells"] / ns
    nrec = recomputed_steps(info, nt)
    per_grad = {"step": nt + nrec, "adj": nt}
    bytes_of = dict(zip(("step", "adj"), kernel_bytes(exec_, info, nt)))
    out = []
    for k in ("step", "adj"):
        ms, n = prof[k]
        if not n:
            continue
        name, bpc = KERNELS[(exec_, k)], bytes_of[k]
        if exec_ == "batched":
            kind = info["stencil"] if k == "step" else info["adj_stencil"]
            tile = (info["tile_x"], info["tile_z"]) if k == "step" else (info["adj_tile_x"], info["adj_tile_z"])
            staging = {1: "per-thread loads", 2: "TMA", 3: "TMA, cell pairs",
                       4: "TMA, cell pairs, staged stores"}.get(kind, "?")
            if k == "step" and kind >= 2 and info["layout"] == 3:
                staging += ", halo ring as single cells"
            if k == "adj" and kind == 1 and info["adj_persistent"]:
                staging += ", persistent grid"
            if k == "adj" and kind == 2 and info.get("adj_layout", 0) >= 2:
                staging += ", cell pairs" + (", 512 threads" if info["adj_layout"] == 3 else "")
            if k == "adj" and info.get("adj_form", 1) == 2:
                staging = "scaled-stress form, " + staging
            name = f"{name.split(' ')[0]} [{staging}, tile {tile[0]}x{tile[1]}] {' '.join(name.split(' ')[1:])}"
        avg = ms / n / 1e3
        achieved = bpc * cells / avg / 1e9
        traffic = None
        if exec_ == "batched":
            key = (k, info["stencil"] if k == "step" else info["adj_stencil"],
                   info["tile_x"] if k == "step" else info["adj_tile_x"],
                   info["tile_z"] if k == "step" else info["adj_tile_z"])
            if k == "step" and info["stencil"] >= 2:
                key = key + (info["layout"], info["staged_stores"])
            if k == "adj":
                key = key + ((info["adj_persistent"],) if info["adj_stencil"] == 1 else (info.get("adj_layout", 0),)) + \
                    (info.get("adj_form", 1),)
            key = key + (info.get("snap_store", 0),)
            t = TRAFFIC_PER_CELL.get(key)
            if isinstance(t, dict):
                n_pass = 0 if info["ckpt_interval"] >= nt else nt - info["stored_steps"]
                if n_pass == 0 or "pass" in t:
                    t = (t.get("pass", 0.0) * n_pass + t["keep"] * (nt + nrec - n_pass)) / (nt + nrec)
                else:
                    t = None
            if t is not None:
                traffic = t * cells
        out.append({"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                    "frac_nominal": achieved / NOMINAL_HBM_GBS,
                    "traffic": traffic, "frac_traffic": None if traffic is None else traffic / avg / 1e9 / hbm,
                    "kernel": name, "bytes_per_cell": bpc, "cells_per_launch": cells,
                    "peak_kind": peak_kind, "launches_timed": n, "avg_us": avg * 1e6,
                    "time_share_est": avg * per_grad[k]})
    tot = sum(r["time_share_est"] for r in out) or 1.0
    for r in out:
        r["time_share_est"] = r["time_share_est"] / tot
    out.sort(key=lambda r: -r["time_share_est"])
    return (out + [None, None])[:2]


def _one_shot_sample(acq, s, nsteps):
    """The oracle's sample: shot s of acq alone, its gradient over nsteps steps."""
    import copy
    a = copy.deepcopy(acq)
    lo, hi = int(a.tr_ptr[s]), int(a.tr_ptr[s + 1])
    a.tr_ptr = np.array([0, hi - lo], np.int32)
    a.ch_xz, a.ch_t = a.ch_xz[lo:hi], a.ch_t[lo:hi]
    a.src_xz, a.mt = a.src_xz[s:s + 1], a.mt[s:s + 1]
    a.nt = nsteps
    a.wavelet = acq.wavelet[s:s + 1, :nsteps + 1]
    return a


def _oracle_worker(job):
    """One process of the all-cores baseline (spawned): the oracle gradient of one
    shot's sample; returns its seconds."""
    acq, vp, vs, rho = job
    from oracle import elastic as E
    t0 = time.perf_counter()
    E.gradient(acq, vp[None], vs[None], rho[None], np.full((acq.ntr, acq.nt), 1e-12))
    return time.perf_counter() - t0


def cpu_baseline(p, budget_s=15.0):
    """The FP64 oracle on the host cores: the gradient of one shot on the full grid
    for a bounded number of steps (a sample of the same workload), first on one
    core (the step count doubles until the sample takes about budget_s / 4), then
    the same sample on as many different shots as there are cores, one spawned
    process each, all at once.  The value is the all-cores throughput."""
    from oracle import elastic as E
    nsteps = 8
    while True:
        a = _one_shot_sample(p.acq, 0, nsteps)
        t0 = time.perf_counter()
        E.gradient(a, p.vp[:1], p.vs[:1], p.rho[:1], np.full((a.ntr, nsteps), 1e-12))
        el = time.perf_counter() - t0
        if el > budget_s / 4 or nsteps >= 4096:
            break
        nsteps *= 2
    cells = p.acq.nx * p.acq.nz * nsteps
    one = {"value": cells / el / 1e9, "cores": 1, "seconds": el}
    import multiprocessing as mp
    ncores = os.cpu_count() or 1
    jobs = [(_one_shot_sample(p.acq, k % p.acq.ns, nsteps), np.asarray(p.vp[k % p.acq.ns]),
             np.asarray(p.vs[k % p.acq.ns]), np.asarray(p.rho[k % p.acq.ns])) for k in range(ncores)]
    try:
        with mp.get_context("spawn").Pool(ncores) as pool:
            pool.map(_oracle_worker, [(_one_shot_sample(p.acq, 0, 2), *[np.asarray(m[0]) for m in (p.vp, p.vs, p.rho)])] * ncores)
            t0 = time.perf_counter()
            pool.map(_oracle_worker, jobs, chunksize=1)
            wall = time.perf_counter() - t0
    except Exception as e:                      # no process pool on this host: the one-core figure stands
        return {"value": one["value"], "unit": UNIT, "cores": 1, "kind": "oracle", "seconds": el, "one_core": one,
                "sample": f"FP64 numpy oracle gradient of one shot on the full 1000x300 grid for {nsteps} steps "
                          f"({el:.1f} s, one core; the all-cores run failed: {type(e).__name__})"}
    return {"value": ncores * cells / wall / 1e9, "unit": UNIT, "cores": ncores, "kind": "oracle",
            "sample": f"FP64 numpy oracle gradient of one shot on the full 1000x300 grid for {nsteps} steps, "
                      f"{ncores} shots at once in {ncores} spawned processes ({wall:.1f} s); one core alone: "
                      f"{one['value']:.4g} G/s ({el:.1f} s)",
            "seconds": wall, "one_core": one}


def run_reference(args):
    rank, world, _ = rank_info()
    if rank != 0:
        return
    p = problem(args.ns, args.nt)
    t_steps = []
    for k in range(args.warmup + args.steps):
        r = cpu_baseline(p, budget_s=8.0)
        if k >= args.warmup:
            t_steps.append(r["value"])
    value = float(np.median(t_steps))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "l2": "n/a (host)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": r["cores"], "kind": "oracle", "sample": r["sample"],
                             "one_core": r["one_core"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def aggregate(ms, cells_per_rank, steps, world, device="cuda"):
    """Whole-job figures from this rank's timed milliseconds: the time is the
    maximum over ranks (every rank waits at the barrier for the slowest), and
    the value counts the cell-updates of all ranks (weak scaling: each rank
    runs its own copy of the workload).  Returns (ms, s per gradient, G/s)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    s = ms / 1e3 / steps
    return ms, s, cells_per_rank * world / s / 1e9


def reduced_storage(efwi, acq, m, d_obs, zoi, eta, ref, plain_s, args):
    """The same workload with FP16 checkpoints and FP16 forward-velocity snapshots,
    every step stored when it fits the device (no recompute): seconds per gradient
    (data term + consistency term, as the headline step), its kernels' rooflines and
    its error against the FP32 path's outputs (ref: phi, g_vp, g_vs, g_rho)."""
    import torch
    ns = acq.ns
    plan = efwi.Plan(acq, exec="batched", ckpt_store="fp16", snap_store="fp16", ckpt_interval="auto")
    b, bp, sink = zoi
    g = tuple(torch.empty_like(m[0]) for _ in range(3))

    def step():
        phi, *_ = plan.gradient(*m, d_obs, out=g)
        for mm, gm, e in zip(m, g, eta):
            plan.regularization_grad(mm, b, bp, sink, e, g=gm)
        return phi

    for _ in range(2):
        step()
    torch.cuda.synchronize()
    plan.prof_enable(97)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = max(2, min(args.steps, 5))
    e0.record(stream)
    for _ in range(steps):
        phi = step()
    e1.record(stream)
    torch.cuda.synchronize()
    s_grad = e0.elapsed_time(e1) / 1e3 / steps
    prof = {k: plan.prof_read(k) for k in ("step", "adj")}
    plan.prof_enable(0)
    info = plan.info()
    rel = lambda a, r: float(torch.linalg.vector_norm((a - r).double()) / torch.linalg.vector_norm(r.double()))
    errs = {"phi": abs(float(phi.item()) - float(ref[0].item())) / abs(float(ref[0].item())),
            "g_vp": rel(g[0], ref[1]), "g_vs": rel(g[1], ref[2]), "g_rho": rel(g[2], ref[3])}
    cells = ns * acq.nx * acq.nz * acq.nt
    roofs = roofline("batched", info, prof, acq.nt, ns)
    out = {"config": {"ckpt_store": "fp16", "snap_store": "fp16", "ckpt_interval": info["ckpt_interval"],
                      "stored_steps": info["stored_steps"], "schedule": schedule_name(info, acq.nt)},
           "steps": steps, "s_per_gradient": s_grad, "value": cells / s_grad / 1e9, "unit": UNIT,
           "speedup_vs_plain_fp32": None if plain_s is None else plain_s / s_grad,
           "rel_err_vs_fp32_path": errs, "roofline": roofs[0], "roofline_other": roofs[1],
           "gradient_roofline": gradient_roofline(info, acq.nt, s_grad), "workspace_GB": info["workspace_bytes"] / 1e9}
    plan.close()
    return out


def sqrt_schedule(efwi, acq, m, d_obs, zoi, eta, ref, args):
    """The headline step on the plain sqrt(nt) schedule (every segment recomputed,
    no step kept by the forward pass): seconds per gradient, and whether its outputs
    equal the headline schedule's bit for bit (ref: phi, g_vp, g_vs, g_rho)."""
    import torch
    plan = efwi.Plan(acq, exec="batched", ckpt_store=args.ckpt_store, snap_store=args.snap_store,
                     ckpt_interval=0, overlap=args.overlap, adj_form=args.adj_form)
    b, bp, sink = zoi
    g = tuple(torch.empty_like(m[0]) for _ in range(3))

    def step():
        phi, *_ = plan.gradient(*m, d_obs, out=g)
        for mm, gm, e in zip(m, g, eta):
            plan.regularization_grad(mm, b, bp, sink, e, g=gm)
        return phi

    step()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = max(2, min(args.steps, 3))
    e0.record(stream)
    for _ in range(steps):
        phi = step()
    e1.record(stream)
    torch.cuda.synchronize()
    s_grad = e0.elapsed_time(e1) / 1e3 / steps
    info = plan.info()
    same = bool(torch.equal(phi, ref[0]) and all(torch.equal(a, r) for a, r in zip(g, ref[1:])))
    out = {"schedule": schedule_name(info, acq.nt), "ckpt_interval": info["ckpt_interval"], "steps": steps,
           "s_per_gradient": s_grad, "value": acq.ns * acq.nx * acq.nz * acq.nt / s_grad / 1e9, "unit": UNIT,
           "outputs_bitwise_equal_to_headline": same, "workspace_GB": info["workspace_bytes"] / 1e9}
    plan.close()
    return out


# objective evaluations the timed l-BFGS iteration of the 4000x1200 record may spend
# (one evaluation = every timed group's gradient, about 15 s per group)
FULL_ITERATION_MAX_LS = 5
# strength of the consistency term in that iteration (the paper sets eta high enough to
# keep the components consistent; see the rule where it is applied)
ETA_HAT = 10.0


def full_iteration(efwi, args):
    """The 4000x1200 extended problem (128 sources with seeded source errors, 1500
    channels, nt = 8000, FP16 checkpoints and snapshots) in groups of 8 shots through
    one plan.  Timed: (a) the plan, created once, and its rebinding from the host;
    (b) the objective of the first `groups` groups and one l-BFGS iteration
    (direction, strong-Wolfe line search, pair update) of the extended objective
    (eq. 8) over the components of those groups, its line search run on the device
    from a CUDA graph (efwi_lbfgs_iterate_device over a device-resident group set, no
    host synchronisation inside the search; its first call captures and instantiates
    the graph, timed apart); (c) the l-BFGS direction over the whole 3 x 128 x 4.8 M
    vector with 5 stored pairs.  With all 16 groups the figures are the configuration's
    own; otherwise the 128-source objective (data term of every component and the
    consistency term) and iteration are 16 / groups times the timed ones (every group
    runs the same kernels on the same shapes).
    Observed data: the timed groups' error-free sources modelled in the true model."""
    import torch
    import workloads as W
    from paper_2305_14130_gb300.groups import GroupSet, group_acquisition
    from paper_2305_14130_gb300.optim import LBFGS
    t_gen = time.perf_counter()
    p = W.full_iteration_4000x1200()
    acq = p.acq
    acq.wavelet = np.asarray(acq.wavelet, np.float32).astype(np.float64)
    t_gen = time.perf_counter() - t_gen
    ns, nz, nx, nt = acq.ns, acq.nz, acq.nx, acq.nt
    gsize = 8
    ngroups = ns // gsize
    G = max(1, min(args.full_iteration_groups, ngroups))
    nsub = G * gsize
    ev = lambda: torch.cuda.Event(enable_timing=True)
    acqs = [group_acquisition(acq, list(range(k * gsize, (k + 1) * gsize)))[0] for k in range(G)]
    dev = lambda a: torch.tensor(np.asarray(a, np.float32), device="cuda")
    t0 = time.perf_counter()
    plan = efwi.Plan(acqs[0], exec="batched", ckpt_store="fp16", snap_store="fp16")
    torch.cuda.synchronize()
    create_s = time.perf_counter() - t0
    info = plan.info()
    out = {"workload": "full_iteration_4000x1200: 128 MT sources with seeded errors (amplitude, shift, rotation), "
                       "1500 DAS ch (0.5 m, 10 m gauge), nt=8000, dt=0.05ms, dx=0.5m; groups of 8 shots",
           "precision": "FP32 stepping, FP16 checkpoints, FP16 snapshots", "ckpt_interval": info["ckpt_interval"],
           "groups_total": ngroups, "groups_timed": G, "plan_create_s": create_s,
           "group_workspace_GB": info["workspace_bytes"] / 1e9,
           "observed_data": "modelled with the error-free sources in the true model", "generate_s": t_gen}
    try:
        x = torch.empty((3, nsub, nz, nx), device="cuda")
        for k, v in enumerate((p.vp, p.vs, p.rho)):
            x[k].copy_(dev(v[0])[None].expand(nsub, nz, nx))
        # observed data: the timed groups' error-free sources in the true model (+4 % Vp / +6 % Vs anomaly)
        d_obs = torch.empty((G, int(acqs[0].tr_ptr[-1]), nt), device="cuda")
        true_wav = np.asarray(p.meta["true_wavelet"], np.float32).astype(np.float64)
        for k in range(G):
            sh = list(range(k * gsize, (k + 1) * gsize))
            tacq = dataclasses.replace(acqs[k], mt=np.asarray(p.meta["true_mt"])[sh], wavelet=true_wav[sh])
            plan.rebind(tacq)
            tm = [dev(v)[None].expand(gsize, nz, nx).contiguous() for v in (p.true_vp, p.true_vs, p.true_rho)]
            plan.forward(*tm, out=d_obs[k])
            del tm
        zsub = type(p.zoi)(**{f: (np.asarray(getattr(p.zoi, f))[:nsub] if np.ndim(getattr(p.zoi, f)) else
                                  getattr(p.zoi, f)) for f in p.zoi.__dataclass_fields__})
        b, bp, sink = efwi.zoi_weights(nsub, nx, nz, acq.dx, acq.dz, zsub)
        gs = GroupSet(plan, acqs)
        # (a) binding the plan to a group from the host (efwi_plan_rebind)
        rebind = []
        for k in range(min(G, 2)):
            t = time.perf_counter()
            plan.rebind(acqs[k])
            torch.cuda.synchronize()
            rebind.append(time.perf_counter() - t)
        # (b) one l-BFGS iteration with the line search on the device
        grad = torch.empty_like(x)
        phi = torch.empty((), dtype=torch.float64, device="cuda")
        a_, b_ = ev(), ev()
        a_.record()
        gs.objective(x, d_obs, p.eta, b, bp, sink, phi=phi, g=grad)
        b_.record()
        b_.synchronize()
        objective_s = a_.elapsed_time(b_) / 1e3
        # the iteration's consistency weights, scale-free: eta_p = ETA_HAT sqrt(2 phi_d(m0)) / ||m_p0||,
        # so that an inconsistency of a fraction delta of the model costs ETA_HAT^2 delta^2 times
        # the starting data misfit (the starting components are equal: phi = phi_d there)
        phi_d0 = float(phi.item())
        eta = tuple(ETA_HAT * (2.0 * phi_d0) ** 0.5 / float(torch.linalg.vector_norm(x[k].double()))
                    for k in range(3))
        gs.objective(x, d_obs, eta, b, bp, sink, phi=phi, g=grad)
        opt = LBFGS(x.numel(), m=5, max_ls=FULL_ITERATION_MAX_LS)
        xf, gf = x.view(-1), grad.view(-1)
        # first trial along d = -g: the largest change of any model value is 1 % of the
        # largest model value (||a d|| = 0.01 max|x| ||g|| / max|g|)
        gmax = float(gf.abs().max())
        if gmax > 0 and np.isfinite(gmax):
            opt.set_step0(0.01 * float(xf.abs().max()) * float(torch.linalg.vector_norm(gf.double())) / gmax)
        dobj = gs.device_objective(d_obs, eta, b, bp, sink)
        phi_start = float(phi.item())
        t = time.perf_counter()
        it = opt.iterate_device(xf, phi, gf, dobj)
        torch.cuda.synchronize()
        first_s = time.perf_counter() - t
        opt.close()
        gs.close()
        del x, grad, d_obs, b, bp, sink
    finally:
        plan.close()
    # (c) the l-BFGS direction over the full vector
    n = 3 * ns * nz * nx
    opt = LBFGS(n, m=5)
    gen = torch.Generator(device="cuda").manual_seed(3)
    sv = torch.empty(n, device="cuda")
    yv = torch.empty(n, device="cuda")
    for _ in range(5):
        sv.normal_(generator=gen)
        yv.copy_(sv).mul_(2.0).add_(torch.randn(n, device="cuda", generator=gen), alpha=0.1)
        opt.push(sv, yv)
    gfull = sv
    opt.direction(gfull)
    torch.cuda.synchronize()
    a_, b_ = ev(), ev()
    a_.record()
    d = opt.direction(gfull)
    b_.record()
    b_.synchronize()
    lbfgs_s = a_.elapsed_time(b_) / 1e3
    del d, sv, yv, gfull
    opt.close()
    scale = ngroups / G
    grad128 = objective_s * scale
    cells = ns * nx * nz * nt
    out.update({
        "rebind_s": rebind, "objective_s_timed_groups": objective_s, "objective_s_per_group": objective_s / G,
        "device_iteration": {"evals": it["evals"], "alpha": it["alpha"], "rate": it["rate"],
                             "ls_failed": it["ls_failed"], "max_ls": FULL_ITERATION_MAX_LS,
                             "phi_before": phi_start, "phi_after": it["phi"], "eta": list(eta),
                             "eta_rule": f"{ETA_HAT} sqrt(2 phi_d(m0)) / ||m_p0|| per parameter field",
                             "first_trial": "largest model change 1 % of max |x|",
                             "s_timed_groups": first_s,
                             "line_search": "on the device (conditional while-node of a CUDA graph); this first "
                                            "call also captures and instantiates the graph"},
        "lbfgs_direction_s_full_vector": lbfgs_s, "lbfgs_n": n,
        "s_per_gradient_128": grad128,
        "s_per_iteration_128": it["evals"] * grad128 + lbfgs_s,
        "per_128_kind": "measured (all groups)" if G == ngroups else
                        f"{ngroups} / {G} x the timed groups (same kernels and shapes in every group)",
        "Gcell_updates_s": cells / grad128 / 1e9})
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist
    rank, world, local = rank_info()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    import __graft_entry__
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    import paper_2305_14130_gb300 as efwi

    p = problem(args.ns, args.nt)
    acq = p.acq
    dev = lambda a, dt=np.float32: torch.tensor(np.asarray(a, dt), device="cuda")
    vp, vs, rho = dev(p.vp), dev(p.vs), dev(p.rho)
    tile = tuple(int(v) for v in args.tile.lower().split("x"))
    adj_tile = tuple(int(v) for v in args.adj_tile.lower().split("x"))
    plan = efwi.Plan(acq, exec=args.exec, ckpt_store=args.ckpt_store, stencil=args.stencil, tile=tile,
                     adj_stencil=args.adj_stencil, adj_tile=adj_tile, overlap=args.overlap,
                     snap_store=args.snap_store, ckpt_interval=args.ckpt if args.ckpt == "auto" else int(args.ckpt),
                     stored_steps=args.stored_steps, adj_form=args.adj_form)
    # observed data: the same sources in the model with the Gaussian anomaly
    ns = acq.ns
    tv = lambda m: dev(np.repeat(np.asarray(m)[None], ns, 0))
    d_obs = plan.forward(tv(p.true_vp), tv(p.true_vs), tv(p.true_rho))
    b, bp, sink = efwi.zoi_weights(ns, acq.nx, acq.nz, acq.dx, acq.dz, p.zoi)
    eta = p.eta
    g = tuple(torch.empty_like(vp) for _ in range(3))
    stream = torch.cuda.current_stream()

    def step():
        phi, gvp, gvs, grho = plan.gradient(vp, vs, rho, d_obs, out=g)
        for m, gm, e in zip((vp, vs, rho), g, eta):
            plan.regularization_grad(m, b, bp, sink, e, g=gm)
        return phi

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # kernels of one step: those the gradient call launched (counted by the plan)
    # plus two per regularization call
    plan.gradient(vp, vs, rho, d_obs, out=g)
    launches_per_step = plan.info()["launches"] + 3 * 2
    torch.cuda.synchronize()

    clocks = Clocks(local)
    plan.prof_enable(97)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ck = clocks.stop()
    ms = e0.elapsed_time(e1)
    prof = {k: plan.prof_read(k) for k in ("step", "adj")}
    plan.prof_enable(0)
    cells = ns * acq.nx * acq.nz * acq.nt
    ms, s_per_grad, value = aggregate(ms, cells, args.steps, world)
    info = plan.info()
    roofs = roofline(args.exec, info, prof, acq.nt, ns)

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        h_vp, h_vs, h_rho = (t.cpu().pin_memory() for t in (vp, vs, rho))
        h_obs = d_obs.cpu().pin_memory()
        h_g = [torch.empty(vp.shape, dtype=torch.float32).pin_memory() for _ in range(3)]
        h_phi = torch.empty((), dtype=torch.float64).pin_memory()
        dvp, dvs, drho, dobs = (torch.empty_like(t) for t in (vp, vs, rho, d_obs))
        h2d = sum(t.numel() * 4 for t in (h_vp, h_vs, h_rho, h_obs))
        d2h = 3 * vp.numel() * 4 + 8

        def e2e_step():
            for d_, h_ in ((dvp, h_vp), (dvs, h_vs), (drho, h_rho), (dobs, h_obs)):
                d_.copy_(h_, non_blocking=True)
            phi, a, b_, c = plan.gradient(dvp, dvs, drho, dobs, out=g)
            for m, gm, e in zip((dvp, dvs, drho), g, eta):
                plan.regularization_grad(m, b, bp, sink, e, g=gm)
            for h_, d_ in zip(h_g, g):
                h_.copy_(d_, non_blocking=True)
            h_phi.copy_(phi, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        n_e2e = max(1, min(args.steps, 2))
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            e2e_step()
        torch.cuda.synchronize()
        el = (time.perf_counter() - t0) / n_e2e
        e2e = {"value": cells * world / el / 1e9, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "s_per_gradient": el}

    # the FP32 path's outputs, for the reduced-storage record's errors
    ref = plan.gradient(vp, vs, rho, d_obs)             # (phi, g_vp, g_vs, g_rho), fresh tensors
    for m, gm, e in zip((vp, vs, rho), ref[1:], eta):
        plan.regularization_grad(m, b, bp, sink, e, g=gm)
    torch.cuda.synchronize()
    plan.close()

    plain = None
    if not args.no_plain and args.exec == "batched":
        pl = efwi.Plan(acq, exec="plain")
        gp = tuple(torch.empty_like(vp) for _ in range(3))
        pl.gradient(vp, vs, rho, d_obs, out=gp)
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        pl.gradient(vp, vs, rho, d_obs, out=gp)
        for m, gm, e in zip((vp, vs, rho), gp, eta):
            pl.regularization_grad(m, b, bp, sink, e, g=gm)
        a1.record(stream)
        torch.cuda.synchronize()
        sp = a0.elapsed_time(a1) / 1e3
        rel = float(torch.linalg.vector_norm(gp[0] - g[0]) / torch.linalg.vector_norm(g[0]))
        plain = {"s_per_gradient": sp, "value": cells / sp / 1e9, "speedup": sp / s_per_grad,
                 "grad_vp_rel_diff": rel}
        pl.close()

    sqrt_rec = None
    if world == 1 and not args.no_sqrt and args.exec == "batched" and info["ckpt_interval"] < acq.nt \
            and info["stored_steps"] > 0:
        sqrt_rec = sqrt_schedule(efwi, acq, (vp, vs, rho), d_obs, (b, bp, sink), eta, ref, args)
        sqrt_rec["headline_speedup"] = sqrt_rec["s_per_gradient"] / s_per_grad

    reduced = None
    if world == 1 and not args.no_reduced and args.exec == "batched":
        reduced = reduced_storage(efwi, acq, (vp, vs, rho), d_obs, (b, bp, sink), eta, ref,
                                  plain["s_per_gradient"] if plain else None, args)
        reduced["speedup_vs_fp32_path"] = s_per_grad / reduced["s_per_gradient"]
    del ref, g, d_obs, b, bp, sink
    full_it = None
    if world == 1 and args.full_iteration_groups > 0 and args.exec == "batched":
        torch.cuda.empty_cache()
        full_it = full_iteration(efwi, args)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(p)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "exec": args.exec, "ckpt_store": args.ckpt_store,
                           "snap_store": args.snap_store,
                           "ckpt_interval": info["ckpt_interval"], "stored_steps": info["stored_steps"],
                           "schedule": schedule_name(info, acq.nt), "tile": [info["tile_x"], info["tile_z"]],
                           "adj_tile": [info["adj_tile_x"], info["adj_tile_z"]],
                           "stencil": {1: "loads", 2: "tma", 3: "tma_pairs", 4: "tma_staged"}.get(info["stencil"], "?"), "stages": info["stages"], "layout": info["layout"],
                           "adj_stencil": {1: "loads", 2: "tma"}.get(info["adj_stencil"], "?"),
                           "adj_form": {1: "stress", 2: "scaled"}.get(info["adj_form"], "?"),
                           "adj_stages": info["adj_stages"], "l2_prefetch": info["prefetch"],
                           "overlap_blocks_per_sm": [info["overlap_fwd_blocks"], info["overlap_adj_blocks"]],
                           "l2": "working set > L2 (wavefields, checkpoints, data >> 129 MB)",
                           "parallelism": f"replicas x{world} (independent extended problems)"},
                "s_per_gradient": s_per_grad,
                "padded_Gcell_updates_s": info["padded_cells"] * acq.nt * world / s_per_grad / 1e9,
                "gpu_launches": launches_per_step * args.steps, "clocks": ck, "roofline": roofs[0],
                "roofline_other": roofs[1],
                "gradient_roofline": gradient_roofline(info, acq.nt, s_per_grad),
                "e2e": e2e, "plain_fp32": plain, "cpu_baseline": cpu,
                "workspace_GB": info["workspace_bytes"] / 1e9,
                "sqrt_schedule": sqrt_rec, "reduced_storage": reduced, "full_iteration": full_it}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

#!/usr/bin/env python3
"""Benchmark: cell-updates/s per SSP-RK3 step of the relativistic-hydro path.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cuda|reference]

Workload: the paper's run (Fig. 3 caption): 256^3 cells, dx = 0.1 fm,
dt = 0.02 fm/c, p = e/3, ellipsoidal-flow start at t0 = 1 fm/c with one jet
from (-8, 0, 0) fm along +x (synthetic, seeded).  A step is one full RK3 step
(three stages, each an x, y and z flux sweep, source and stage combination).

The headline line is the FP64 path (the one held to 1e-10 of the FP64
oracle); FP32 and mixed precision are reported under "variants" with their
measured error against the FP64 path.  Timing: W untimed warm-up steps, then
K steps bracketed by a barrier and device synchronisation, CUDA events on the
library's stream; the state (671 MB per copy in FP64) is larger than L2, so
no flush is needed.  With --gpus N > 1 (torchrun) every rank runs an
independent replica (the path is not sharded) and the time is the max over
ranks.

--impl reference times the FP64 CPU oracle on the host cores instead (one RK3
step of a 128^3 sub-grid of the same workload per bench step).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s per RK3 step at 256^3 (FP64 vs FP32); % of HBM roofline"
UNIT = "cell-updates/s"

# Algorithmic work per cell of one directional sweep of one RK3 stage (FLOPs
# with FMA = 2, division and square root = 1), counted on the textbook
# evaluation: one interface is the LLF split (5 x 14 FMAs + alpha/2 = 141), 10
# WENO7 reconstructions of 122 (candidates 28, differences 15, A 20, B 4,
# beta 32, weights 23) and the 5 flux sums, 1366 in all; the x sweep adds the
# flux difference (10), the primitive recovery (23), |v|^2 (5), rho_x (14) and
# F_x (10); y and z add difference and accumulation (15), rho_d and F_d; z adds
# the stage combination (20, averaged over the three stages).
FLOP_PER_INTERFACE = 141 + 10 * 122 + 5
FLOP_PER_CELL = {"sweep_x": FLOP_PER_INTERFACE + 10 + 23 + 5 + 14 + 10,
                 "sweep_y": FLOP_PER_INTERFACE + 15 + 14 + 10,
                 "sweep_z": FLOP_PER_INTERFACE + 15 + 14 + 10 + 20}
FLOP_PER_CELL_STEP = 3 * sum(FLOP_PER_CELL.values())
# Algorithmic HBM bytes per cell per step: 40 field accesses (stage 1 reads 5 and
# writes 5; stages 2 and 3 read 10 and write 5) in storage precision.
FIELD_ACCESSES_PER_CELL_STEP = 40

# DRAM bytes per cell per sweep launch, from ncu captures of the 256^3 workload
# (dram__bytes_read.sum + dram__bytes_write.sum, mean over the three stages of a step),
# taken with the kernels as built; a kernel change makes them stale, and a stale entry
# is None (reported as null).  The FP64 sweeps changed their reciprocal after the last
# capture (loads and stores unchanged: 77.4 / 117.6 / 145.3 B per cell before).
TRAFFIC_B_PER_CELL = {
    ("fp64", "sweep_x"): None, ("fp64", "sweep_y"): None, ("fp64", "sweep_z"): None,
    ("fp32", "sweep_x"): 37.5, ("fp32", "sweep_y"): 57.7, ("fp32", "sweep_z"): 71.9,
    ("mixed", "sweep_x"): 58.3, ("mixed", "sweep_y"): 78.3, ("mixed", "sweep_z"): 124.8,
}

# Peaks for an ALU-bound path, derived from unit counts and clocks: 148 SMs x
# 128 FP32 lanes x 2 FLOP/FMA x 2.032 GHz; FP64 takes the nominal B300 rate.
PEAK_FP32_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12
PEAK_FP64_TFLOPS = 1.25


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, 0
    import torch
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    if backend == "nccl":
        torch.cuda.set_device(local)
    dist.init_process_group(backend=backend)
    return rank, ws, local


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(x: float, ws: int) -> float:
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() and dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """Samples SM clock, power and throttle reasons with nvidia-smi every 200 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id: str | None):
        self.bus_id = bus_id
        self.proc = None
        self.lines = []

    def __enter__(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.bus_id:
            cmd += ["-i", self.bus_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def _bus_id():
    try:
        import torch
        p = torch.cuda.get_device_properties(torch.cuda.current_device())
        return "%08x:%02x:%02x.0" % (p.pci_domain_id, p.pci_bus_id, p.pci_device_id)
    except Exception:
        return None


_GRID = 256


def _workload():
    from paper_1511_02137_b300 import workloads as W
    if _GRID == 256:
        return W.ELLIPSOIDAL_256
    return W.scaled(W.ELLIPSOIDAL_256, _GRID)


def _make_ctx(hy, w, precision, prim_host):
    cfg = hy.hydro_config_default(*w.n, precision=precision, dx=w.dx, dt=w.dt, t0=w.t0)
    ctx = hy.hydro_create(cfg)
    hy.hydro_set_initial(ctx, hy.HYDRO_PRIMITIVE, prim_host)
    for j in w.jets:
        hy.hydro_add_jet(ctx, j.x0, j.direction, j.t_start)
    return ctx


def _time_device(hy, ctx, steps, warmup, ws, sampler_bus=None):
    """Device-resident timing; returns (seconds, per-kernel profile, clocks)."""
    import torch
    stream = ctx.stream
    hy.hydro_step(ctx, warmup)
    hy.hydro_profile_enable(ctx, True)
    _barrier(ws)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(sampler_bus) as clk:
        ev0.record(stream)
        hy.hydro_step(ctx, steps)
        ev1.record(stream)
        ev1.synchronize()
    torch.cuda.synchronize()
    _barrier(ws)
    sec = ev0.elapsed_time(ev1) / 1e3
    prof = {}
    for k, name in ((hy.HYDRO_KERNEL_SWEEP_X, "sweep_x"), (hy.HYDRO_KERNEL_SWEEP_Y, "sweep_y"),
                    (hy.HYDRO_KERNEL_SWEEP_Z, "sweep_z")):
        ms, n = hy.hydro_profile_query(ctx, k)
        prof[name] = {"ms": ms, "launches": n}
    hy.hydro_profile_enable(ctx, False)
    return sec, prof, clk.summary()


def _roofline(prof, cells, precision):
    dom = max(prof, key=lambda k: prof[k]["ms"])
    p = prof[dom]
    avg_s = p["ms"] / 1e3 / max(p["launches"], 1)
    flop = cells * FLOP_PER_CELL[dom]
    achieved = flop / avg_s / 1e12
    peak = PEAK_FP64_TFLOPS if precision == "fp64" else PEAK_FP32_TFLOPS
    total_ms = sum(v["ms"] for v in prof.values())
    return {"bound": "alu", "kernel": dom, "achieved": round(achieved, 4), "peak": round(peak, 3),
            "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
            "traffic": (TRAFFIC_B_PER_CELL[(precision, dom)] * cells
                        if TRAFFIC_B_PER_CELL.get((precision, dom)) is not None else None),
            "peak_source": ("nominal B300 FP64 rate (profiling recipe)" if precision == "fp64" else
                            "derived: 148 SMs x 128 FP32 lanes x 2 x 2.032 GHz"),
            "flop_per_launch": flop, "avg_launch_ms": round(avg_s * 1e3, 4),
            "share": {k: round(v["ms"] / total_ms, 4) for k, v in prof.items()}}


def _hbm(sec, steps, cells, precision):
    byte = 4 if precision == "fp32" else 8
    gbs = cells * steps * FIELD_ACCESSES_PER_CELL_STEP * byte / sec / 1e9
    peak = _peaks().get("hbm_gbs", 6400.0)
    return {"algorithmic_GBps": round(gbs, 1), "peak_GBps": peak, "frac_of_measured_hbm": round(gbs / peak, 4),
            "frac_of_8TBps": round(gbs / 8000.0, 4)}


def _e2e(hy, w, prim_pinned, out_pinned, steps):
    """Same metric through the public C ABI with host buffers: H2D of the initial
    state, `steps` calls of hydro_step(ctx, 1) (each reads the step status back),
    D2H of the final fields, all inside the wall-clock timed region."""
    import torch
    cfg = hy.hydro_config_default(*w.n, precision="fp64", dx=w.dx, dt=w.dt, t0=w.t0)
    ctx = hy.hydro_create(cfg)
    for j in w.jets:
        hy.hydro_add_jet(ctx, j.x0, j.direction, j.t_start)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hy.hydro_set_initial(ctx, hy.HYDRO_PRIMITIVE, prim_pinned)
    for _ in range(steps):
        hy.hydro_step(ctx, 1)
    hy.hydro_read_fields(ctx, hy.HYDRO_CONSERVED, out_pinned)
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    hy.hydro_destroy(ctx)
    state_bytes = 5 * w.cells * 8
    diag_bytes = 256   # per-step status/diagnostics block read back by hydro_step
    return sec, state_bytes, diag_bytes


def _cpu_baseline(w, seconds_hint=20.0):
    """The FP64 oracle as it stands, on all host cores: one RK3 step of the
    workload (the full 256^3 grid)."""
    import oracle
    from paper_1511_02137_b300 import workloads as W
    threads = oracle.max_threads()
    U = oracle.prim_to_cons(W.ellipsoidal_primitives(w))
    cfg = oracle.Config(*w.n, dx=w.dx, dt=w.dt, t0=w.t0)
    jets = [oracle.Jet(j.x0, j.direction, j.t_start) for j in w.jets]
    t0 = time.perf_counter()
    oracle.run(cfg, U, 1, jets)
    sec = time.perf_counter() - t0
    return {"value": w.cells / sec, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"1 RK3 step of the full {w.n[0]}x{w.n[1]}x{w.n[2]} workload, FP64, {threads} OpenMP threads",
            "seconds": round(sec, 2)}


def _batched(hy, steps, warmup):
    """The batched configuration: 64 uneven grids (edges 64-160), FP32, tiles
    picked by the autotuner, steps replayed from a CUDA graph.  Wall clock around
    the synchronous hydro_batch_step call (host jet tables, graph launch, sync)."""
    import torch
    from paper_1511_02137_b300 import workloads as W
    E = W.ENSEMBLE_64
    cfg = hy.hydro_config_default(1, 1, 1, precision="fp32")
    b = hy.hydro_batch_create(cfg, [w.n for w in E.events])
    for e, w in enumerate(E.events):
        hy.hydro_batch_set_initial(b, e, hy.HYDRO_PRIMITIVE, W.ellipsoidal_primitives(w).ravel())
        for j in w.jets:
            hy.hydro_batch_add_jet(b, e, j.x0, j.direction, j.t_start)
    choice, ms = hy.hydro_batch_autotune(b)
    hy.hydro_batch_step(b, warmup)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hy.hydro_batch_step(b, steps)
    sec = time.perf_counter() - t0
    hy.hydro_batch_destroy(b)
    cells = E.cells
    names = ["sweep_x", "sweep_y", "sweep_z"]
    per = {names[d]: ms[d][choice[d]] for d in range(3)}
    dom = max(per, key=per.get)
    achieved = FLOP_PER_CELL[dom] * cells / (per[dom] / 1e3) / 1e12
    return {"workload": E.name, "events": len(E.events), "cells": cells, "precision": "fp32",
            "value": cells * steps / sec, "unit": UNIT, "ms_per_step": sec * 1e3 / steps, "steps": steps,
            "tile_choice": {names[d]: choice[d] for d in range(3)},
            "autotune_ms": {names[d]: ms[d] for d in range(3)},
            "roofline": {"bound": "alu", "kernel": dom, "achieved": round(achieved, 4),
                         "peak": round(PEAK_FP32_TFLOPS, 3), "unit": "TFLOP/s",
                         "frac": round(achieved / PEAK_FP32_TFLOPS, 4),
                         "note": "per-launch time of the chosen tile shape from the autotuner (first-stage sweep)"},
            "timing": "wall clock around hydro_batch_step (CUDA graph replay, includes host jet tables and sync)"}


def _adjoint_one(hy, grid, steps, precision):
    import torch
    from paper_1511_02137_b300 import adjoint as A
    from paper_1511_02137_b300 import workloads as W
    jet = W.JetSpec((-4.0, 0.0, 0.0), (1.0, 0.0, 0.0), 1.0)
    w = W.Workload(name=f"ellipsoidal-flow {grid}^3, {steps} RK3 steps, 1 jet (adjoint)", n=(grid, grid, grid),
                   steps=steps, sigma=(4.0, 5.0, 6.0), jets=(jet,))
    prim = W.ellipsoidal_primitives(w)
    run = A.ConeEnergyRun(hy.hydro_config_default(*w.n, precision=precision), w.steps, min(10, w.steps), w.jets,
                          torch.from_numpy(prim[1:].copy()).cuda(), apex=jet.x0, axis=jet.direction)
    e = torch.from_numpy(prim[0].copy()).cuda()
    kr = torch.tensor(4.0, dtype=torch.float64, requires_grad=True)
    kc = torch.tensor(2.5, dtype=torch.float64, requires_grad=True)
    A.cone_energy(e, kr.detach(), kc.detach(), run)            # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    A.cone_energy(e, kr.detach(), kc.detach(), run)
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    ev = e.clone().requires_grad_(True)
    t0 = time.perf_counter()
    J = A.cone_energy(ev, kr, kc, run)
    J.backward()
    torch.cuda.synchronize()
    t_all = time.perf_counter() - t0
    res = {"workload": w.name, "precision": precision, "checkpoint_every": min(10, w.steps), "J_GeV": J.item(),
           "dJ_dk_rad": kr.grad.item(), "dJ_dk_coll": kc.grad.item(),
           "forward_s": round(t_fwd, 3), "backward_s": round(t_all - t_fwd, 3),
           "backward_over_forward": round((t_all - t_fwd) / t_fwd, 3),
           "forward_cell_updates_per_s": w.cells * w.steps / t_fwd}
    return res, ev.grad


def _adjoint(hy, grid=128, steps=50):
    """The adjoint configuration: 128^3, 50 steps, checkpoint every 10, one jet
    from (-4, 0, 0) fm along +x, energy in a 30-degree cone of radius 3 fm around
    the jet axis; gradient with respect to k_rad, k_coll and e(x), in FP64 and in
    mixed precision.  Times one forward and one forward + backward through
    torch.autograd (wall clock, synced).  The mixed entry carries its gradient's
    deviation from the FP64 gradient (relative, max-norm for the e field)."""
    out, g64 = _adjoint_one(hy, grid, steps, "fp64")
    mixed, g32 = _adjoint_one(hy, grid, steps, "mixed")
    mixed["vs_fp64"] = {"J": abs(mixed["J_GeV"] / out["J_GeV"] - 1),
                        "dJ_dk_rad": abs(mixed["dJ_dk_rad"] / out["dJ_dk_rad"] - 1),
                        "dJ_dk_coll": abs(mixed["dJ_dk_coll"] / out["dJ_dk_coll"] - 1),
                        "dJ_de_maxnorm": float((g32 - g64).abs().max() / g64.abs().max())}
    out["mixed"] = mixed
    return out


def run_cuda(args, rank, ws):
    import numpy as np
    import torch

    from paper_1511_02137_b300 import build
    build.build()
    from paper_1511_02137_b300 import hydro as hy
    from paper_1511_02137_b300 import workloads as W

    w = _workload()
    prim = W.ellipsoidal_primitives(w).ravel()
    prim_pinned = torch.from_numpy(prim).pin_memory()
    out_pinned = torch.empty(5 * w.cells, dtype=torch.float64).pin_memory()
    bus = _bus_id()

    results = {}
    finals = {}
    launches = 0
    for prec in args.precisions:
        ctx = _make_ctx(hy, w, prec, prim_pinned)
        sec, prof, clk = _time_device(hy, ctx, args.steps, args.warmup, ws, bus)
        sec = _max_over_ranks(sec, ws)
        diag = hy.hydro_get_diag(ctx)
        finals[prec] = hy.hydro_read_fields(ctx, hy.HYDRO_CONSERVED)
        hy.hydro_destroy(ctx)
        del ctx
        launches = sum(v["launches"] for v in prof.values()) if prec == args.precisions[0] else launches
        results[prec] = {"sec": sec, "prof": prof, "clocks": clk, "diag": diag}

    head = args.precisions[0]
    r = results[head]
    cells = w.cells
    value = cells * args.steps * ws / r["sec"]
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": r["sec"] * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32", "mixed": "f64+f32"}[head],
        "data": "synthetic (seeded ellipsoidal-flow initial state and jet, no dataset)",
        "config": {"workload": w.name, "grid": list(w.n), "dx_fm": w.dx, "dt_fm_per_c": w.dt, "t0_fm_per_c": w.t0,
                   "precision": head, "weno_order": 7, "parallelism": "replicas" if ws > 1 else "single GPU",
                   "l2": "no flush: one FP64 state copy is 671 MB > 126 MB L2"},
        "roofline": _roofline(r["prof"], cells, head),
        "hbm": _hbm(r["sec"], args.steps, cells, head),
        "gpu_launches": launches,
        "clocks": r["clocks"],
    }
    variants = {}
    for prec in args.precisions[1:]:
        v = results[prec]
        ref = finals.get("fp64")
        err = None
        if ref is not None:
            a = finals[prec].reshape(5, -1)
            b = ref.reshape(5, -1)
            err = [float(x) for x in np.abs(a - b).max(axis=1) / np.abs(b).max(axis=1)]
        variants[prec] = {"value": cells * args.steps * ws / v["sec"], "ms_per_step": v["sec"] * 1e3 / args.steps,
                          "speedup_vs_fp64": results["fp64"]["sec"] / v["sec"] if "fp64" in results else None,
                          "err_vs_fp64_per_field_E_Mx_My_Mz_R": err,
                          "roofline": _roofline(v["prof"], cells, prec), "hbm": _hbm(v["sec"], args.steps, cells, prec),
                          "clocks": v["clocks"]}
    out["variants"] = variants
    if not args.no_batched:
        out["batched"] = _batched(hy, args.steps, args.warmup)
    if not args.no_adjoint:
        out["adjoint"] = _adjoint(hy, args.adjoint_grid, args.adjoint_steps)
    if not args.no_e2e:
        sec, sb, db = _e2e(hy, w, prim_pinned, out_pinned, args.steps)
        sec = _max_over_ranks(sec, ws)
        out["e2e"] = {"value": cells * args.steps * ws / sec, "unit": UNIT,
                      "h2d_bytes_per_step": sb / args.steps, "d2h_bytes_per_step": sb / args.steps + db,
                      "note": "initial state uploaded and final fields read back once per run of K steps; "
                              "hydro_step(ctx, 1) per step reads its status block"}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = _cpu_baseline(w)
    elif rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = None
    return out


def run_reference(args, rank, ws):
    """The FP64 oracle on the host cores, one RK3 step of a 128^3 sub-grid of the
    workload per bench step."""
    if rank != 0:
        return None
    import oracle
    from paper_1511_02137_b300 import workloads as W
    oracle.build()
    w = W.scaled(_workload(), 128, steps=1)
    U = oracle.prim_to_cons(W.ellipsoidal_primitives(w))
    cfg = oracle.Config(*w.n, dx=w.dx, dt=w.dt, t0=w.t0)
    jets = [oracle.Jet(j.x0, j.direction, j.t_start) for j in w.jets]
    for s in range(args.warmup):
        U, _ = oracle.run(cfg, U, 1, jets, step0=s)
    t0 = time.perf_counter()
    for s in range(args.steps):
        U, _ = oracle.run(cfg, U, 1, jets, step0=args.warmup + s)
    sec = time.perf_counter() - t0
    value = w.cells * args.steps / sec
    threads = oracle.max_threads()
    sample = (f"1 RK3 step of the 128^3 centre sub-grid of the 256^3 workload per bench step, FP64 oracle, "
              f"{threads} OpenMP threads")
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": sec * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic (seeded ellipsoidal-flow initial state)", "impl": "reference",
            "config": {"workload": _workload().name, "grid": list(_workload().n), "precision": "fp64",
                       "sample": "128^3 sub-grid"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["cuda", "reference"], default="cuda")
    ap.add_argument("--precisions", default="fp64,fp32,mixed",
                    help="comma list; the first is the headline line, fp64 must come first for error columns")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 64-event batched ensemble measurement")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the 128^3 adjoint timing")
    ap.add_argument("--adjoint-only", action="store_true",
                    help="run only the adjoint section (for profiling its kernels)")
    ap.add_argument("--adjoint-grid", type=int, default=128)
    ap.add_argument("--adjoint-steps", type=int, default=50)
    ap.add_argument("--grid", type=int, default=256,
                    help="cube edge; 256 is the paper's run, smaller edges are centre sub-grids for profiling")
    args = ap.parse_args(argv)
    global _GRID
    _GRID = args.grid
    args.precisions = [p.strip() for p in args.precisions.split(",") if p.strip()]
    args.warmup = max(args.warmup, 3)   # timing rule: at least 3 untimed warm-up steps
    rank, ws, _ = _dist()
    if args.adjoint_only:
        from paper_1511_02137_b300 import build
        build.build()
        from paper_1511_02137_b300 import hydro as hy
        out = {"adjoint": _adjoint(hy, args.adjoint_grid, args.adjoint_steps)} if rank == 0 else None
    elif args.impl == "reference":
        out = run_reference(args, rank, ws)
    else:
        out = run_cuda(args, rank, ws)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

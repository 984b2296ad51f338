#!/usr/bin/env python3
"""Benchmark: cell-updates/s per SSP-RK3 step of the relativistic-hydro path.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cuda|reference]

Workload: the paper's run (Fig. 3 caption): 256^3 cells, dx = 0.1 fm,
dt = 0.02 fm/c, p = e/3, ellipsoidal-flow start at t0 = 1 fm/c with one jet
from (-8, 0, 0) fm along +x (synthetic, seeded).  A step is one full RK3 step
(three stages, each an x, y and z flux sweep, source and stage combination).

The headline line is the FP64 path (the one held to 1e-10 of the FP64
oracle); FP32 and mixed precision are reported under "variants" (the last key
of the line), each timed on its own run and with its error per field against
the FP64 path on the mixed-precision configuration (256^3, 3 seeded jets, 70
steps).  Timing: W untimed warm-up steps, then K steps bracketed by a barrier
and device synchronisation, CUDA events on the library's stream; the state
(671 MB per copy in FP64) is larger than L2, so no flush is needed.  Clocks
are sampled through NVML every 25 ms during each timed region.  The ALU
peaks that the roofline fractions divide by are measured in the same run by
FMA-throughput kernels (hydro_alu_peak).  With --gpus N > 1 (torchrun) every
rank runs an independent replica (the path is not sharded) and the time is
the max over ranks.  The line also carries "e2e" (the same steps through the
C ABI from pinned host buffers, copies included), "cpu_baseline" (the oracle
on the host cores), "adjoint" (128^3 x 50 steps, backward / forward cost),
"batched" (the 64-event ensemble) and "weno5" (the WENO5 variant of the
workload), each with its own roofline where it has one.

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
# with FMA = 2, division and square root = 1), counted on the canonical
# evaluation of each term: one interface is the LLF split (5 fields x 14 FMAs +
# alpha/2 = 141), 10 WENO7 reconstructions of 122 (candidates 28, differences
# 15, A 20, B 4, beta 32, weights 23) and the 5 flux sums, 1366 in all; the x
# sweep adds the flux difference (10), the primitive recovery (21), |v|^2 (5),
# rho_x (12) and F_x / 2 (10); y and z add difference and accumulation (15),
# rho_d and F_d / 2; z adds the stage combination (20, averaged over the three
# stages).
FLOP_RECON_W7 = 122
FLOP_RECON_W5 = 65
FLOP_SPLIT, FLOP_FSUM = 141, 5
FLOP_DIFF, FLOP_DIFF_ACC, FLOP_STAGE = 10, 15, 20
FLOP_C2P, FLOP_V2, FLOP_RHO, FLOP_HALF_FLUX = 21, 5, 12, 10
FLOP_PER_INTERFACE = FLOP_SPLIT + 10 * FLOP_RECON_W7 + FLOP_FSUM
FLOP_PER_CELL = {
    "sweep_x": FLOP_PER_INTERFACE + FLOP_DIFF + FLOP_C2P + FLOP_V2 + FLOP_RHO + FLOP_HALF_FLUX,
    "sweep_y": FLOP_PER_INTERFACE + FLOP_DIFF_ACC + FLOP_RHO + FLOP_HALF_FLUX,
    "sweep_z": FLOP_PER_INTERFACE + FLOP_DIFF_ACC + FLOP_RHO + FLOP_HALF_FLUX + FLOP_STAGE}
FLOP_PER_CELL_STEP = 3 * sum(FLOP_PER_CELL.values())
# The same count for the WENO5 variant: the split over 5 cells per side (5 x 10
# FMAs + alpha/2 = 101), 10 WENO5 reconstructions of 65 (candidates 15, second
# differences 9, first-derivative terms 9, beta 15, weights 17) and the 5 flux
# sums, 756 per interface; the per-cell terms as for WENO7.
FLOP_PER_INTERFACE_W5 = 101 + 10 * FLOP_RECON_W5 + 5
FLOP_PER_CELL_W5 = {k: v - FLOP_PER_INTERFACE + FLOP_PER_INTERFACE_W5 for k, v in FLOP_PER_CELL.items()}
# Algorithmic HBM bytes per cell per step: 40 field accesses (stage 1 reads 5 and
# writes 5; stages 2 and 3 read 10 and write 5) in storage precision.
FIELD_ACCESSES_PER_CELL_STEP = 40

# DRAM bytes per cell per sweep launch, from ncu captures of the 256^3 workload
# (dram__bytes_read.sum + dram__bytes_write.sum, mean over the three stages of a step),
# taken with the kernels as built; a kernel change makes them stale, and a stale entry
# is None (reported as null).
TRAFFIC_B_PER_CELL = {
    ("fp64", "sweep_x"): 116.9, ("fp64", "sweep_y"): 142.2, ("fp64", "sweep_z"): 169.6,
    ("fp32", "sweep_x"): 37.5, ("fp32", "sweep_y"): 57.7, ("fp32", "sweep_z"): 71.9,
    ("mixed", "sweep_x"): 55.2, ("mixed", "sweep_y"): 61.9, ("mixed", "sweep_z"): 132.4,
}

# Fallback peaks for an ALU-bound path, used only when the in-run measurement
# fails: 148 SMs x 128 FP32 lanes x 2 FLOP/FMA x 2.032 GHz, and FP64 at 1/64 of it.
PEAK_FP32_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12
PEAK_FP64_TFLOPS = PEAK_FP32_TFLOPS / 64

# The paper's own performance statement, quoted as context (no number for this metric).
PAPER_CONTEXT = "paper (Sec. 1): its CUDA code ran over 100x faster than the same computation on a CPU; neither GPU nor CPU is named"


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
    """Samples SM clock, power and throttle reasons during a timed region: through
    NVML every 25 ms, or (without NVML) nvidia-smi every 100 ms.  Each sample is
    one line in nvidia-smi's CSV layout (sm MHz, max sm MHz, W, reasons bitmask,
    hw_slowdown, hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap)."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    # NVML clock-event reason bits: hw_slowdown, hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap
    BITS = (0x8, 0x40, 0x20, 0x4)

    def __init__(self, bus_id: str | None, period_s: float = 0.025):
        self.bus_id = bus_id
        self.period = period_s
        self.proc = None
        self.thread = None
        self.stop = threading.Event()
        self.lines = []

    def __enter__(self):
        try:
            import pynvml
            pynvml.nvmlInit()
            h = (pynvml.nvmlDeviceGetHandleByPciBusId(self.bus_id) if self.bus_id
                 else pynvml.nvmlDeviceGetHandleByIndex(0))
            self.thread = threading.Thread(target=self._poll_nvml, args=(pynvml, h), daemon=True)
            self.thread.start()
            return self
        except Exception:
            pass
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100"]
        if self.bus_id:
            cmd += ["-i", self.bus_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _poll_nvml(self, nv, h):
        smax = nv.nvmlDeviceGetMaxClockInfo(h, nv.NVML_CLOCK_SM)
        while not self.stop.is_set():
            try:
                sm = nv.nvmlDeviceGetClockInfo(h, nv.NVML_CLOCK_SM)
                pw = nv.nvmlDeviceGetPowerUsage(h) / 1000.0
                r = nv.nvmlDeviceGetCurrentClocksEventReasons(h)
                flags = ", ".join("Active" if r & b else "Not Active" for b in self.BITS)
                self.lines.append(f"{sm}, {smax}, {pw:.1f}, {r:#x}, {flags}")
            except Exception:
                pass
            self.stop.wait(self.period)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        self.stop.set()
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
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


def _make_ctx(hy, w, precision, prim_host, order=7):
    cfg = hy.hydro_config_default(*w.n, precision=precision, dx=w.dx, dt=w.dt, t0=w.t0, weno_order=order)
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


def _roofline(prof, cells, precision, peaks=None, order=7):
    """Roofline of the dominant sweep: algorithmic FLOPs per launch over its mean
    CUDA-event launch time, against the measured FMA peak of the flux type (FP64
    for the FP64 path, FP32 for FP32 and mixed).  DRAM traffic from the ncu table
    (WENO7 only)."""
    dom = max(prof, key=lambda k: prof[k]["ms"])
    p = prof[dom]
    avg_s = p["ms"] / 1e3 / max(p["launches"], 1)
    flop = cells * (FLOP_PER_CELL if order == 7 else FLOP_PER_CELL_W5)[dom]
    achieved = flop / avg_s / 1e12
    key = "fp64_tflops" if precision == "fp64" else "fp32_tflops"
    if peaks and peaks.get(key):
        peak = peaks[key]
        source = f"measured in this run: {peaks['method']}"
    else:
        peak = PEAK_FP64_TFLOPS if precision == "fp64" else PEAK_FP32_TFLOPS
        source = "derived: 148 SMs x 128 FP32 lanes x 2 x 2.032 GHz (FP64: 1/64 of it)"
    total_ms = sum(v["ms"] for v in prof.values())
    return {"bound": "alu", "kernel": dom, "achieved": round(achieved, 4), "peak": round(peak, 3),
            "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
            "traffic": (TRAFFIC_B_PER_CELL[(precision, dom)] * cells
                        if order == 7 and TRAFFIC_B_PER_CELL.get((precision, dom)) is not None else None),
            "peak_source": source, "flop_per_launch": flop, "avg_launch_ms": round(avg_s * 1e3, 4),
            "share": {k: round(v["ms"] / total_ms, 4) for k, v in prof.items()}}


def _alu_peaks(hy, bus):
    """FMA throughput of this GPU measured now: the best of two launches of each
    FMA-chain kernel (FP32 FFMA, packed FP32x2 FFMA2, FP64 DFMA), ~0.4 s each, with
    the SM clock sampled during them."""
    import torch
    kinds = (("ffma", hy.HYDRO_PEAK_FFMA, 6_000_000), ("ffma2", hy.HYDRO_PEAK_FFMA2, 3_000_000),
             ("dfma", hy.HYDRO_PEAK_DFMA, 90_000))
    res = {}
    try:
        with ClockSampler(bus) as clk:
            for name, kind, iters in kinds:
                hy.hydro_alu_peak(kind, max(1, iters // 50))   # warm-up
                best = 0.0
                for _ in range(2):
                    flop, ms = hy.hydro_alu_peak(kind, iters)
                    best = max(best, flop / (ms / 1e3) / 1e12)
                res[name] = round(best, 3)
        torch.cuda.synchronize()
    except Exception as exc:   # report, and fall back to the derived peaks
        return {"error": str(exc)[:120]}
    c = clk.summary()
    return {"fp32_tflops": max(res["ffma"], res["ffma2"]), "fp64_tflops": res["dfma"],
            "ffma_tflops": res["ffma"], "ffma2_tflops": res["ffma2"], "dfma_tflops": res["dfma"],
            "sm_mhz": c["sm_mhz"], "reasons": c["reasons"], "samples": c["samples"],
            "method": "8 independent FMA chains per thread on every SM (hydro_alu_peak), best of 2"}


def _hbm(sec, steps, cells, precision):
    byte = 4 if precision == "fp32" else 8
    gbs = cells * steps * FIELD_ACCESSES_PER_CELL_STEP * byte / sec / 1e9
    peak = _peaks().get("hbm_gbs", 6400.0)
    return {"algorithmic_GBps": round(gbs, 1), "peak_GBps": peak, "frac_of_measured_hbm": round(gbs / peak, 4),
            "frac_of_8TBps": round(gbs / 8000.0, 4)}


def _err_per_field(a, b):
    a = a.reshape(5, -1)
    b = b.reshape(5, -1)
    import numpy as np
    return [float("%.3g" % x) for x in np.abs(a - b).max(axis=1) / np.abs(b).max(axis=1)]


def _e2e(hy, w, prim_pinned, out_pinned, steps, precision="fp64"):
    """Same metric through the public C ABI with host buffers: H2D of the initial
    state, `steps` calls of hydro_step(ctx, 1) (each reads the step status back),
    D2H of the final fields, all inside the wall-clock timed region."""
    import torch
    cfg = hy.hydro_config_default(*w.n, precision=precision, dx=w.dx, dt=w.dt, t0=w.t0)
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


def _cpu_baseline(w, single_core_grid=96):
    """The FP64 oracle as it stands: one RK3 step of the workload (the full 256^3
    grid) on all host cores, and one step of the centre sub-grid of edge
    `single_core_grid` on one core, whose per-cell rate is extrapolated (not run)
    to the full workload's steps."""
    import oracle
    from paper_1511_02137_b300 import workloads as W
    threads = oracle.max_threads()
    jets = [oracle.Jet(j.x0, j.direction, j.t_start) for j in w.jets]
    U = oracle.prim_to_cons(W.ellipsoidal_primitives(w))
    cfg = oracle.Config(*w.n, dx=w.dx, dt=w.dt, t0=w.t0)
    t0 = time.perf_counter()
    oracle.run(cfg, U, 1, jets)
    sec = time.perf_counter() - t0
    out = {"value": w.cells / sec, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"1 RK3 step of the full {w.n[0]}x{w.n[1]}x{w.n[2]} workload, FP64, {threads} OpenMP threads",
           "seconds": round(sec, 2)}
    ws = W.scaled(w, single_core_grid, steps=1)
    U1 = oracle.prim_to_cons(W.ellipsoidal_primitives(ws))
    cfg1 = oracle.Config(*ws.n, dx=ws.dx, dt=ws.dt, t0=ws.t0, nthreads=1)
    t0 = time.perf_counter()
    oracle.run(cfg1, U1, 1, jets)
    sec1 = time.perf_counter() - t0
    rate1 = ws.cells / sec1
    out["single_core"] = {
        "value": rate1, "unit": UNIT, "cores": 1, "kind": "oracle",
        "sample": f"1 RK3 step of the {single_core_grid}^3 centre sub-grid, FP64, 1 thread",
        "seconds": round(sec1, 2),
        "full_run_s_extrapolated": round(w.cells * w.steps / rate1, 1),
        "full_run": f"{w.steps} steps of {w.n[0]}^3 at this per-cell rate: extrapolated, not run"}
    return out


def _batched(hy, steps, warmup, peaks=None, events=None, edge=None):
    """The batched configuration: 64 uneven grids (edges 64-160), FP32, tiles
    picked by the autotuner, steps replayed from a CUDA graph.  Wall clock around
    the synchronous hydro_batch_step call (host jet tables, graph launch, sync).
    For profiling: `events` keeps the first events of the ensemble, `edge` replaces
    every grid by one cube of that edge (the first event's profile)."""
    import torch
    from paper_1511_02137_b300 import workloads as W
    E = W.ENSEMBLE_64
    if events:
        E = W.Ensemble(name=f"{E.name} [first {events} events]", events=E.events[:events], steps=E.steps)
    if edge:
        E = W.Ensemble(name=f"{E.name} [{len(E.events)} x {edge}^3]",
                       events=tuple(W.replace(w, n=(edge, edge, edge)) for w in E.events), steps=E.steps)
    cfg = hy.hydro_config_default(1, 1, 1, precision="fp32")
    b = hy.hydro_batch_create(cfg, [w.n for w in E.events])
    for e, w in enumerate(E.events):
        hy.hydro_batch_set_initial(b, e, hy.HYDRO_PRIMITIVE, W.ellipsoidal_primitives(w).ravel())
        for j in w.jets:
            hy.hydro_batch_add_jet(b, e, j.x0, j.direction, j.t_start)
    choice, ms = hy.hydro_batch_autotune(b)
    _, per_tile = hy.hydro_batch_get_tuning(b)
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
    peak = (peaks or {}).get("fp32_tflops") or PEAK_FP32_TFLOPS
    return {"workload": E.name, "events": len(E.events), "cells": cells, "precision": "fp32",
            "value": cells * steps / sec, "unit": UNIT, "ms_per_step": round(sec * 1e3 / steps, 3), "steps": steps,
            "tile_choice": [choice[d] for d in range(3)],
            "launch_per_tile": [per_tile[d] for d in range(3)],
            "autotune_ms": [[round(x, 3) for x in ms[d]] for d in range(3)],
            "roofline": {"bound": "alu", "kernel": dom, "achieved": round(achieved, 4), "peak": round(peak, 3),
                         "unit": "TFLOP/s", "frac": round(achieved / peak, 4)},
            "timing": "wall clock around hydro_batch_step (graph replay); roofline from the autotuner's launch"}


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
    A.cone_energy(e, torch.tensor(4.0, dtype=torch.float64), torch.tensor(2.5, dtype=torch.float64), run)   # warm-up
    # three calls of forward + backward, CUDA events on the library stream (torch's
    # current stream); medians of the forward and backward times and of the per-call ratio
    fwd, bwd, ratio = [], [], []
    for _ in range(3):
        ev = e.clone().requires_grad_(True)
        kr = torch.tensor(4.0, dtype=torch.float64, requires_grad=True)
        kc = torch.tensor(2.5, dtype=torch.float64, requires_grad=True)
        mark = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        torch.cuda.synchronize()
        mark[0].record()
        J = A.cone_energy(ev, kr, kc, run)
        mark[1].record()
        J.backward()
        mark[2].record()
        mark[2].synchronize()
        f, b = mark[0].elapsed_time(mark[1]) / 1e3, mark[1].elapsed_time(mark[2]) / 1e3
        fwd.append(f)
        bwd.append(b)
        ratio.append(b / f)
    res = {"precision": precision, "checkpoint_every": min(10, w.steps), "J_GeV": J.item(),
           "dJ_dk_rad": kr.grad.item(), "dJ_dk_coll": kc.grad.item(),
           "forward_s": round(statistics.median(fwd), 5), "backward_s": round(statistics.median(bwd), 5),
           "backward_over_forward": round(statistics.median(ratio), 3),
           "timing": "medians of 3 calls, CUDA events"}
    return res, ev.grad


def _adjoint(hy, grid=128, steps=50):
    """The adjoint configuration: 128^3, 50 steps, checkpoint every 10, one jet
    from (-4, 0, 0) fm along +x, energy in a 30-degree cone of radius 3 fm around
    the jet axis; gradient with respect to k_rad, k_coll and e(x), in FP64 and in
    mixed precision.  Times three calls of forward and backward through
    torch.autograd (CUDA events on the library stream, medians).  The mixed entry
    carries its gradient's deviation from the FP64 gradient (relative, max-norm
    for the e field)."""
    out, g64 = _adjoint_one(hy, grid, steps, "fp64")
    mixed, g32 = _adjoint_one(hy, grid, steps, "mixed")
    mixed["vs_fp64"] = {"J": float("%.3g" % abs(mixed["J_GeV"] / out["J_GeV"] - 1)),
                        "dJ_dk_rad": float("%.3g" % abs(mixed["dJ_dk_rad"] / out["dJ_dk_rad"] - 1)),
                        "dJ_dk_coll": float("%.3g" % abs(mixed["dJ_dk_coll"] / out["dJ_dk_coll"] - 1)),
                        "dJ_de_maxnorm": float("%.3g" % float((g32 - g64).abs().max() / g64.abs().max()))}
    out["workload"] = f"ellipsoidal-flow {grid}^3, {steps} RK3 steps, 1 jet, cone 30 deg r < 3 fm"
    out["mixed"] = mixed
    return out


def _weno5(hy, w, prim, args, ws, bus, peaks):
    """The WENO5 variant of the step on the headline workload, each precision of
    the run: W warm-up steps, then K steps (FP64) or max(K, 100) (FP32, mixed),
    CUDA events on the library stream, the dominant sweep against the measured
    FMA peak with the WENO5 FLOP count."""
    res = {}
    for prec in args.precisions:
        steps = args.steps if prec == "fp64" else max(args.steps, 100)
        ctx = _make_ctx(hy, w, prec, prim, order=5)
        sec, prof, clk = _time_device(hy, ctx, steps, args.warmup, ws, bus)
        sec = _max_over_ranks(sec, ws)
        hy.hydro_destroy(ctx)
        roof = _roofline(prof, w.cells, prec, peaks, order=5)
        res[prec] = {"value": w.cells * steps * ws / sec, "ms_per_step": round(sec * 1e3 / steps, 4), "steps": steps,
                     "roofline": {k: roof[k] for k in ("kernel", "achieved", "peak", "frac", "avg_launch_ms",
                                                       "share")},
                     "flop_per_cell_step": 3 * sum(FLOP_PER_CELL_W5.values()), "clocks": clk}
    res["config"] = f"{w.name}, weno_order 5, same workload and timing as the WENO7 lines"
    return res


def _variant(hy, W, prec, args, ws, bus, peaks, ref_final, pinned=None):
    """One reduced-precision variant on the mixed-precision configuration (256^3,
    3 seeded jets): its error per field against the FP64 path after the 70
    configured steps, then the timing of a fresh run (W warm-up steps, then
    max(K, 300) steps so that the clock sampler sees the timed region), and the
    same metric end to end through the C ABI with host buffers (K steps; pinned =
    the pinned host buffers of the initial state and the read-back)."""
    w = W.ELLIPSOIDAL_256_3JETS if _GRID == 256 else W.scaled(W.ELLIPSOIDAL_256_3JETS, _GRID)
    prim = W.ellipsoidal_primitives(w).ravel()
    err = None
    if ref_final is not None:
        ctx = _make_ctx(hy, w, prec, prim)
        hy.hydro_step(ctx, w.steps)
        err = _err_per_field(hy.hydro_read_fields(ctx, hy.HYDRO_CONSERVED), ref_final)
        hy.hydro_destroy(ctx)
    steps = max(args.steps, args.variant_steps)
    ctx = _make_ctx(hy, w, prec, prim)
    sec, prof, clk = _time_device(hy, ctx, steps, args.warmup, ws, bus)
    sec = _max_over_ranks(sec, ws)
    hy.hydro_destroy(ctx)
    roof = _roofline(prof, w.cells, prec, peaks)
    e2e = None
    if pinned is not None and not args.no_e2e:
        esec, sb, db = _e2e(hy, w, pinned[0], pinned[1], args.steps, prec)
        esec = _max_over_ranks(esec, ws)
        e2e = {"value": w.cells * args.steps * ws / esec, "h2d_bytes_per_step": sb / args.steps,
               "d2h_bytes_per_step": sb / args.steps + db}
    return sec, steps, {
        "value": w.cells * steps * ws / sec, "ms_per_step": round(sec * 1e3 / steps, 4), "steps": steps,
        "err_vs_fp64_per_field_E_Mx_My_Mz_R": err,
        "roofline": {k: roof[k] for k in ("kernel", "achieved", "peak", "frac", "traffic", "avg_launch_ms", "share")},
        "hbm": _hbm(sec, steps, w.cells, prec)["frac_of_measured_hbm"], "e2e": e2e, "clocks": clk}


def run_cuda(args, rank, ws):
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
    peaks = _alu_peaks(hy, bus) if not args.no_peaks else {}
    head = args.precisions[0]
    cells = w.cells

    # the headline: device-resident timing of K steps
    ctx = _make_ctx(hy, w, head, prim_pinned)
    sec, prof, clk = _time_device(hy, ctx, args.steps, args.warmup, ws, bus)
    sec = _max_over_ranks(sec, ws)
    hy.hydro_destroy(ctx)
    del ctx
    launches = sum(v["launches"] for v in prof.values())
    value = cells * args.steps * ws / sec
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": sec * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32", "mixed": "f64+f32"}[head],
        "data": "synthetic (seeded ellipsoidal-flow initial state and jet, no dataset)",
        "config": {"workload": w.name, "grid": list(w.n), "dx_fm": w.dx, "dt_fm_per_c": w.dt, "t0_fm_per_c": w.t0,
                   "precision": head, "weno_order": 7, "parallelism": "replicas" if ws > 1 else "single GPU",
                   "l2": "no flush: one FP64 state copy is 671 MB > 126 MB L2"},
        "roofline": _roofline(prof, cells, head, peaks),
    }
    if not args.no_e2e:
        esec, sb, db = _e2e(hy, w, prim_pinned, out_pinned, args.steps, head)
        esec = _max_over_ranks(esec, ws)
        out["e2e"] = {"value": cells * args.steps * ws / esec, "unit": UNIT,
                      "h2d_bytes_per_step": sb / args.steps, "d2h_bytes_per_step": sb / args.steps + db,
                      "note": "state uploaded and read back once per K steps; each step reads its status block"}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = _cpu_baseline(w)
    elif rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = None
    out["clocks"] = clk
    out["gpu_launches"] = launches
    out["peaks"] = peaks
    out["hbm"] = _hbm(sec, args.steps, cells, head)
    out["paper_context"] = PAPER_CONTEXT
    if not args.no_adjoint:
        out["adjoint"] = _adjoint(hy, args.adjoint_grid, args.adjoint_steps)
    if not args.no_batched:
        out["batched"] = _batched(hy, args.steps, args.warmup, peaks)
    if not args.no_weno5:
        out["weno5"] = _weno5(hy, w, prim_pinned, args, ws, bus, peaks)
    # reduced precisions last: their error against the FP64 path on the
    # mixed-precision configuration, their own timing and roofline
    variants = {}
    if len(args.precisions) > 1:
        ref = None
        if head == "fp64" and not args.no_variant_error:
            w3 = W.ELLIPSOIDAL_256_3JETS if _GRID == 256 else W.scaled(W.ELLIPSOIDAL_256_3JETS, _GRID)
            ctx = _make_ctx(hy, w3, "fp64", W.ellipsoidal_primitives(w3).ravel())
            hy.hydro_step(ctx, w3.steps)
            ref = hy.hydro_read_fields(ctx, hy.HYDRO_CONSERVED)
            hy.hydro_destroy(ctx)
        for prec in args.precisions[1:]:
            vsec, vsteps, v = _variant(hy, W, prec, args, ws, bus, peaks, ref,
                                       (prim_pinned, out_pinned) if _GRID == 256 else None)
            v["speedup_vs_fp64"] = round((sec / args.steps) / (vsec / vsteps), 2) if head == "fp64" else None
            variants[prec] = v
        variants["config"] = ("error: 256^3, 3 seeded jets, 70 steps vs the FP64 path (per field, norm-relative); "
                              "timing: same workload, fresh run")
    out["variants"] = variants
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
    ap.add_argument("--no-weno5", action="store_true", help="skip the WENO5 variant timing")
    ap.add_argument("--weno5-only", action="store_true",
                    help="run only the WENO5 section (for profiling its kernels)")
    ap.add_argument("--no-peaks", action="store_true", help="skip the ALU peak measurement (derived peaks instead)")
    ap.add_argument("--no-variant-error", action="store_true",
                    help="skip the 70-step FP64 reference run behind the variants' error columns")
    ap.add_argument("--variant-steps", type=int, default=300, help="timed steps of each reduced-precision variant")
    ap.add_argument("--batched-only", action="store_true",
                    help="run only the batched ensemble section (for profiling its kernels)")
    ap.add_argument("--batched-events", type=int, default=0, help="first N events of the ensemble (profiling)")
    ap.add_argument("--batched-edge", type=int, default=0, help="every event a cube of this edge (profiling)")
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
    if args.batched_only:
        from paper_1511_02137_b300 import build
        build.build()
        from paper_1511_02137_b300 import hydro as hy
        out = ({"batched": _batched(hy, args.steps, args.warmup, None, args.batched_events, args.batched_edge)}
               if rank == 0 else None)
    elif args.adjoint_only:
        from paper_1511_02137_b300 import build
        build.build()
        from paper_1511_02137_b300 import hydro as hy
        out = {"adjoint": _adjoint(hy, args.adjoint_grid, args.adjoint_steps)} if rank == 0 else None
    elif args.weno5_only:
        from paper_1511_02137_b300 import build
        build.build()
        from paper_1511_02137_b300 import hydro as hy
        from paper_1511_02137_b300 import workloads as W
        w = _workload()
        prim = W.ellipsoidal_primitives(w).ravel()
        peaks = _alu_peaks(hy, _bus_id()) if not args.no_peaks else {}
        out = {"weno5": _weno5(hy, w, prim, args, ws, _bus_id(), peaks)}
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

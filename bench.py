#!/usr/bin/env python3
"""Throughput of the GB300 EM-PIC timestep (gather + Boris push + Esirkepov
deposit + Yee update) in particle-steps/s, with the HBM roofline fraction of
the dominant kernel, the end-to-end figure through the C ABI with host
buffers, and the FP64 oracle timed on the host cores as the CPU baseline.

Default workload: 3D laser-wakefield box 256x256x1024 cells (x, y
transverse, z the propagation axis), dx=dy=1, dz=0.3, dt=0.27 c/omega0,
n=0.0025 n_c at 8 particles per cell (536,870,912 electrons), cold, a0=4
laser (waist 60, FWHM 30), open z with a moving window, quadratic shapes,
FP32.  A step is one full timestep of every particle and cell.

    python bench.py [--steps K] [--warmup W] [--impl native|reference]
Under torchrun each rank advances its own replica on its own GPU (the path
has no exchange step on one GPU), timed with a barrier on both sides.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s (gather+push+deposit), % HBM roofline; batched & adjoint vs plain"
UNIT = "particle-steps/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="lwfa_3d",
                    choices=["lwfa_3d", "warm_3d", "thermal_2d", "bunch_3d", "scan_2d", "adjoint_2d", "order_sweep",
                             "frozen_3d"])
    ap.add_argument("--order", type=int, default=0, help="shape order override (warm_3d)")
    ap.add_argument("--adjoint-steps", type=int, default=2000)
    ap.add_argument("--scan-runs", type=int, default=64)
    ap.add_argument("--autotune", action="store_true", help="choose the tuning with the autotuner first")
    ap.add_argument("--scale", type=float, default=1.0, help="shrink every grid axis (debug runs only)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget-s", type=float, default=20.0)
    ap.add_argument("--tuning", default="", help="json dict of pic_tuning overrides")
    ap.add_argument("--out", default="", help="also write the JSON line to this file")
    ap.add_argument("--no-full-run", action="store_true", help="skip the whole-run (500-step) timing")
    ap.add_argument("--no-scan", action="store_true", help="skip the batched-scan ratio")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint ratio")
    ap.add_argument("--scan-steps", type=int, default=40)
    return ap.parse_args()


def workload(name, scale, order=0):
    from paper_1310_0930_gb300 import inputs
    if name == "lwfa_3d":
        n = (256, 256, 1024)
        if scale != 1.0:
            n = tuple(max(16, int(round(v * scale / 8)) * 8) for v in n)
        return inputs.lwfa_3d(n=n)
    if name == "bunch_3d":
        return inputs.bunch_3d()
    if name == "warm_3d":
        # uniform warm plasma (u_th = 0.1, the paper's throughput benchmark,
        # Sec. 4), 256^3 cells at 8 ppc: every particle moves and deposits
        n = tuple(max(16, int(round(256 * scale / 8)) * 8) for _ in range(3))
        w = inputs.thermal_3d(n=n, order=order or 2)
        w.name = "warm_3d"
        w.uth = 0.1
        return w
    return inputs.thermal_2d()


def particle_chunks(w):
    from paper_1310_0930_gb300 import inputs
    if w.dim == 3:
        chunks = list(inputs.background_chunks(w, 64))
    else:
        chunks = [inputs.background(w)]
    if w.bunch is not None:
        chunks.append(inputs.bunch(w))
    return chunks


# Per-slot figures of the particle phase's dominant kernel from an ncu capture
# of a small case of the same workload (summaries in profiles/, named below):
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) and warp
# instructions (smsp__inst_executed.sum) per particle slot the kernel
# processed, scaled to the timed launches by their slot counts (the kernel's
# traffic grows in proportion to its slots).
ZERO_PROFILE = {
    ("lwfa_3d", 2): (16.9, 1.52, "push_zero_kernel_lwfa3d_64x64x256.md"),
}
# the same per live-tile particle for the staged kernel (classification
# included in its events, not in these figures)
STAGED_PROFILE = {
    ("lwfa_3d", 2): (42.7, 32.7, "push_kernel_lwfa3d_quadratic_128x128x512.md"),
}


def aggregate_replicas(elapsed, units):
    """Whole-job figures of independent replicas, one per rank: the slowest
    rank's elapsed time and the units all ranks processed (max and sum over
    the ranks of the initialised process group; the local figures alone
    without one).  Tensors live where the backend wants them (CUDA for nccl,
    host memory for gloo)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(elapsed), float(units)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(elapsed)], dtype=torch.float64, device=dev)
    u = torch.tensor([float(units)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


# A particle slot of a zero-field tile: its packed cell (absorption) and its
# momentum (at rest or not) are read; a particle at rest keeps its state, so
# nothing is written and its offsets are not read.
ZERO_SLOT_BYTES = 4 + 12


def algorithmic_bytes(w, n_particles, streamed=0.0, live_cells=None):
    """Bytes the method must move once per step: per particle of a live tile
    the state read + written, 2 * (4 packed cell + 4*dim offsets + 12
    momentum [+4 weight]); per slot of a zero-field tile (`streamed` of them)
    ZERO_SLOT_BYTES; per cell of a live tile (`live_cells`, default every
    cell) 36 = gather E,B (24) + J write (12); per cell 60 = Yee reads E,B,J
    (36) + writes E,B (24).  The particle phase alone: particles + 36 B per
    live cell."""
    sp = 4 + 4 * w.dim + 12 + (4 if (w.knots is not None or w.bunch is not None) else 0)
    parts = (n_particles - streamed) * 2 * sp + streamed * ZERO_SLOT_BYTES
    cells = w.n_cells if live_cells is None else min(float(w.n_cells), live_cells)
    step = parts + cells * 36 + w.n_cells * 60
    push = parts + cells * 36
    return step, push, sp


def tile_cells(w, tuning):
    """Cells of one tile: the tuning's tile, else the default of the
    dimension (3D 8 x 8 x 8, 2D 16 x 16)."""
    t = (tuning or {}).get("tile")
    if t:
        return int(np.prod(t[: w.dim]))
    return 512 if w.dim == 3 else 256


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.proc = None
        sel = []
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(device_index).uuid)
            sel = ["-i", uuid if uuid.startswith("GPU-") else "GPU-" + uuid]
        except Exception:
            sel = []
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                                          "-lms", "200"] + sel, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.3)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        return parse_clocks(out)


def parse_clocks(text):
    """Clock record from nvidia-smi samples (the fields of Clocks.Q, one line
    per sample, csv without header or units): median SM clock under load,
    the largest maximum clock, the throttle reasons seen active in any
    sample; None without a usable sample."""
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in text.splitlines():
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            mx.append(float(f[2]))
        except ValueError:
            continue
        for nm, v in zip(names, f[5:9]):
            if v.lower().startswith("active"):
                reasons.add(nm)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
            "samples": len(sm)}


def cpu_baseline(w, budget_s, steps=3, warmup=0):
    """Time the FP64 oracle, as it stands, on a bounded crop of the same
    workload (same cells, dt, density, ppc, order, laser) on all host cores:
    `warmup` untimed steps, then `steps` timed steps, the crop sized from a
    one-step calibration so that the timed steps take about budget_s."""
    import oracle
    from paper_1310_0930_gb300 import inputs
    cores = os.cpu_count() or 1

    def make(ncrop):
        c = inputs.Workload(w.name, w.dim, ncrop, w.d, w.dt, w.order, w.ppc, w.density, uth=w.uth,
                            jitter=w.jitter, seed=w.seed, open_last=w.open_last, laser=w.laser, window=w.window)
        parts = inputs.background(c)
        laser = None
        if c.laser is not None:
            L = c.laser
            laser = dict(a0=L.a0, waist=L.waist, fwhm=L.fwhm, plane=L.plane, pol=L.pol, t_peak=L.peak_time())
        sim = oracle.Sim(c.dim, c.n, c.d, c.dt, c.order, open_last=c.open_last, laser=laser, nthreads=cores)
        x = np.zeros((3, parts.n))
        x[: c.dim] = parts.positions64()
        sim.load(x, parts.u.astype(np.float64), parts.w.astype(np.float64))
        return sim, parts.n

    # calibrate on a small crop, then size the sample to the budget
    base = (16, 16, 64) if w.dim == 3 else (32, 32)
    sim, n = make(base)
    t0 = time.perf_counter()
    sim.step(1)
    t_ps = (time.perf_counter() - t0) / n
    target = max(n, int(budget_s / max(t_ps, 1e-9) / max(1, steps)))
    grow = max(1.0, (target / n) ** 0.5)
    if w.dim == 3:
        ncrop = (min(w.n[0], int(16 * grow) // 8 * 8 or 16), min(w.n[1], int(16 * grow) // 8 * 8 or 16), 64)
    else:
        ncrop = (min(w.n[0], int(32 * grow) // 8 * 8), min(w.n[1], int(32 * grow) // 8 * 8))
    sim, n = make(ncrop)
    if warmup:
        sim.step(warmup)
    t0 = time.perf_counter()
    sim.step(steps)
    dt_s = time.perf_counter() - t0
    return {"value": n * steps / dt_s, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "FP64 oracle, %s crop %s cells (%d particles, same d/dt/density/ppc/order/laser), "
                      "%d warm-up + %d timed steps, %.1f s timed" % (w.name, "x".join(map(str, ncrop)), n, warmup,
                                                                     steps, dt_s)}


def workload_config(w, n_particles):
    """The workload description shared by both arms of the JSON line."""
    return {"workload": "%s %s cells, %d ppc, order %d" % (w.name, "x".join(map(str, w.n)), w.ppc_total, w.order),
            "grid": list(w.n), "d": list(w.d), "dt": w.dt, "particles": int(n_particles),
            "window": w.window is not None, "laser_a0": w.laser.a0 if w.laser else None}


def scan_measure(args, steps, warmup, window_moves=False):
    """Batched parameter scan: independent 2D LWFA runs of uneven sizes
    advanced by one handle (one launch per phase over every run's tiles,
    persistent push kernel, CUDA-graph replay) against the same runs advanced
    one after another by plain single-run handles, the same `steps` timed
    steps per run in both.  window_moves: every run's moving window starts a
    quarter of the way into the timed steps, so that both arms time window
    shifts and the injection of new plasma."""
    import torch
    from paper_1310_0930_gb300 import autotune, inputs
    from paper_1310_0930_gb300.sim import Simulation, TorchMemory

    torch.cuda.set_device(0)
    runs = inputs.scan_2d(count=args.scan_runs)
    if window_moves:
        for w in runs:
            w.window.t0 = w.dt * (warmup + steps // 4)
    parts = [inputs.background(w) for w in runs]
    n_total = sum(p.n for p in parts)
    cells = sum(w.n_cells for w in runs)
    tuning = json.loads(args.tuning) if (args.tuning and args.workload == "scan_2d") else {}
    if args.autotune:
        sub = list(range(min(8, len(runs))))

        def loader(sim):
            for i, r in enumerate(sub):
                sim.select(i)
                sim.load(parts[r])
            return sum(parts[r].n for r in sub)
        tuning = autotune.tune([runs[r] for r in sub], loader, refresh=True)

    def timed(sim, clocks=None):
        st = sim.mem.stream
        sim.step(warmup)
        sim.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        sim.step(steps)
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    batch = Simulation(runs, tuning=tuning, memory=TorchMemory())
    for r, p in enumerate(parts):
        batch.select(r)
        batch.load(p)
    clocks = Clocks(0)
    ms_b = timed(batch)
    clk_b = clocks.stop()
    shifts_b = []
    for r in range(len(runs)):
        batch.select(r)
        shifts_b.append(batch.diagnostics()["shifts"])
    batch.close()
    del batch
    single_tuning = {k: v for k, v in tuning.items() if k != "persistent"}
    ms_s = 0.0
    clocks = Clocks(0)
    for w, p in zip(runs, parts):
        sim = Simulation(w, tuning=single_tuning, memory=TorchMemory())
        sim.load(p)
        ms_s += timed(sim)
        sim.close()
    clk_s = clocks.stop()
    value = n_total * steps / (ms_b / 1e3)
    seq = n_total * steps / (ms_s / 1e3)
    return {"runs": len(runs), "particles": n_total, "cells": cells, "steps": steps, "warmup": warmup,
            "tuning": tuning, "window_shifts_per_run": [min(shifts_b), max(shifts_b)],
            "batched": {"value": value, "ms_per_step": ms_b / steps, "clocks": clk_b},
            "sequential_plain": {"value": seq, "ms_per_step": ms_s / steps, "clocks": clk_s},
            "batched_over_sequential": value / seq}


def scan_bench(args):
    """The batched scan as the bench line's own workload."""
    m = scan_measure(args, args.steps, args.warmup)
    line = {"metric": METRIC, "value": m["batched"]["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": m["batched"]["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "scan_2d: %d independent 2D LWFA runs (nz 256-2048 x nx 128-512, dz=0.3, "
                                   "dx=1, dt=0.28, 4-16 ppc, n 0.001-0.01, a0 1-6), quadratic" % m["runs"],
                       "runs": m["runs"], "particles": m["particles"], "cells": m["cells"], "tuning": m["tuning"]},
            "batched": m["batched"], "sequential_plain": m["sequential_plain"],
            "batched_over_sequential": m["batched_over_sequential"], "clocks": m["batched"]["clocks"]}
    print(json.dumps(line), flush=True)
    if args.out:
        with open(args.out, "w") as f:
            f.write(json.dumps(line) + "\n")
    return 0


def adjoint_measure(args, S, warmup):
    """Gradient of the trailing-window kinetic energy with respect to 32
    density knots and a0 on the 2D LWFA box 256 x 1024 cells (dx=1, dz=0.3,
    dt=0.28), 16 ppc, window moving at c from t = 120 (the knots span the
    lab-frame plasma length, box plus window travel), checkpoints every 100
    steps: the plain forward run against the forward run with checkpoints
    plus the reverse sweep."""
    import torch
    from paper_1310_0930_gb300 import inputs
    from paper_1310_0930_gb300.sim import Simulation, TorchMemory

    torch.cuda.set_device(0)
    w = inputs.adjoint_2d(steps=S)
    parts = inputs.background(w)
    obj = (100.0, 300.0, 2.0)

    def wall(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t0, out

    tuning = json.loads(args.tuning) if (args.tuning and args.workload == "adjoint_2d") else None
    plain = Simulation(w, per_particle_weight=True, tuning=tuning, memory=TorchMemory())
    plain.load(parts)
    plain.step(warmup)
    plain.sync()
    clocks = Clocks(0)
    t_fwd, _ = wall(lambda: (plain.step(S), plain.sync()))
    clk_f = clocks.stop()
    plain.close()
    sim = Simulation(w, track_ids=True, per_particle_weight=True, tuning=tuning, memory=TorchMemory())
    sim.load(parts)
    kept = sim.adjoint_begin(S, 100)
    clocks = Clocks(0)
    t_fwd_ck, _ = wall(lambda: (sim.step(S), sim.sync()))
    t_bwd, res = wall(lambda: sim.adjoint_backward(*obj, n_knots=len(w.knots)))
    clk_g = clocks.stop()
    sim.close()
    n = parts.n
    return {"workload": "adjoint_2d: 2D LWFA 256x1024 cells, 16 ppc, 32 density knots, a0=3, %d steps, "
                        "moving window from t=120, checkpoint every 100, gradient w.r.t. knots and a0" % S,
            "particles": n, "steps": S, "tuning": tuning, "forward_s": t_fwd, "forward_clocks": clk_f,
            "forward_with_checkpoints_s": t_fwd_ck, "reverse_s": t_bwd, "gradient_clocks": clk_g,
            "gradient_over_forward": (t_fwd_ck + t_bwd) / t_fwd,
            "segments": {"checkpoints": -(-S // 100), "recorded_by_forward": kept},
            "L": res["L"], "dL_da0": res["dL_da0"], "dL_dknots_norm": float(np.linalg.norm(res["dL_dknots"]))}


def adjoint_bench(args):
    """The adjoint form as the bench line's own workload."""
    S = args.adjoint_steps
    m = adjoint_measure(args, S, args.warmup)
    n = m["particles"]
    line = {"metric": METRIC, "value": n * S / (m["forward_with_checkpoints_s"] + m["reverse_s"]), "unit": UNIT,
            "n_gpus": 1, "steps": S, "warmup": args.warmup,
            "ms_per_step": 1e3 * (m["forward_with_checkpoints_s"] + m["reverse_s"]) / S, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": m["workload"], "particles": n}, "clocks": m["gradient_clocks"]}
    line.update({k: v for k, v in m.items() if k not in ("workload", "particles")})
    print(json.dumps(line), flush=True)
    if args.out:
        with open(args.out, "w") as f:
            f.write(json.dumps(line) + "\n")
    return 0


# Table 3 of the paper: the warm-plasma benchmark (128^3 cells, 8 ppc,
# u_th = 0.1) on one 8-core Intel E5-2680 (AVX, FP32): full PIC step time
# per particle per CPU for interpolation orders 1 to 4, context for the
# per-GPU figure (the quartic per-core entry is garbled in the source; the
# per-CPU time is used).
TABLE3_NS_PER_PARTICLE_PER_CPU = {1: 7.4, 2: 13.6, 3: 24.8, 4: 61.5}


def order_sweep(args):
    """Shape orders 1 to 4 on the warm-plasma benchmark of Table 3: 128^3
    cells, 8 ppc (16,777,216 electrons), u_th = 0.1, periodic, every particle
    moving: particle-steps/s and ns per particle per GPU for each order, the
    push phase's share, and the paper's per-CPU time beside it."""
    import torch
    from paper_1310_0930_gb300 import inputs
    from paper_1310_0930_gb300.sim import Simulation, TorchMemory

    torch.cuda.set_device(0)
    tuning = json.loads(args.tuning) if args.tuning else None
    rows = {}
    for order in (1, 2, 3, 4):
        w = inputs.thermal_3d(n=(128, 128, 128), order=order)
        w.name = "warm_3d"
        w.uth = 0.1
        parts = inputs.background(w)
        mem = TorchMemory()
        sim = Simulation(w, tuning=tuning, memory=mem)
        sim.load(parts)
        sim.step(args.warmup)
        sim.sync()
        clocks = Clocks(0)
        sim.profile_begin(args.steps)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(mem.stream)
        sim.step(args.steps)
        e1.record(mem.stream)
        torch.cuda.synchronize()
        phases, _ = sim.profile_end()
        clk = clocks.stop()
        ms = e0.elapsed_time(e1) / args.steps
        d = sim.diagnostics()
        sim.close()
        n = parts.n
        rows[order] = {"particle_steps_per_s": n / (ms / 1e3), "ms_per_step": ms,
                       "push_ms_per_step": phases["push"] / args.steps,
                       "ns_per_particle": ms * 1e6 / n, "clocks": clk, "status": d["status"],
                       "paper_ns_per_particle_per_cpu": TABLE3_NS_PER_PARTICLE_PER_CPU[order]}
        rows[order]["gpu_over_cpu"] = rows[order]["paper_ns_per_particle_per_cpu"] / rows[order]["ns_per_particle"]
    base = rows[1]["ms_per_step"]
    for order in rows:
        rows[order]["time_over_linear"] = rows[order]["ms_per_step"] / base
    line = {"metric": METRIC, "value": rows[2]["particle_steps_per_s"], "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": rows[2]["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "order_sweep: warm plasma 128^3 cells, 8 ppc, u_th 0.1, periodic, orders 1-4 "
                                   "(value: quadratic)", "particles": 16777216},
            "orders": rows, "clocks": rows[2]["clocks"]}
    print(json.dumps(line), flush=True)
    if args.out:
        with open(args.out, "w") as f:
            f.write(json.dumps(line) + "\n")
    return 0


# Table 2 of the paper: frozen (zero-temperature) plasma on the full Jaguar
# machine, linear (s1) and quadratic (s2) interpolation: 1463.5 and 784.0
# G particles/s at 516.9 and 736.1 TFlop/s, i.e. about 2.7x the operations
# per particle for quadratic at about 1.8x the time.
TABLE2_FROZEN = {"linear_gparts_per_s": 1463.5, "quadratic_gparts_per_s": 784.0,
                 "quadratic_over_linear_time": 1463.5 / 784.0,
                 "quadratic_over_linear_ops": (736.1 / 784.0) / (516.9 / 1463.5)}


def frozen_bench(args):
    """The frozen-plasma asymptotic test of Table 2: a zero-temperature plasma
    (256^3 cells, 8 ppc, 134,217,728 electrons, periodic) at linear and
    quadratic order.  (a) No fields, as in the paper: nothing moves and every
    tile takes the zero-field streaming kernel (the step's asymptotic limit is
    the particle state's HBM traffic).  (b) The same plasma, immobile (mass
    1e30 electron masses) in imposed smooth E and B: every tile is staged and
    every particle gathers E and B and is pushed, but none moves, so no
    current is deposited -- the gather-and-push cost whose order dependence
    the paper's remark on operations and time is about."""
    import torch
    from paper_1310_0930_gb300 import inputs
    from paper_1310_0930_gb300.sim import Simulation, TorchMemory

    torch.cuda.set_device(0)
    n = tuple(max(16, int(round(256 * args.scale / 8)) * 8) for _ in range(3))
    rows = {}
    for case in ("no_fields", "imposed_fields"):
        for order in (1, 2):
            w = inputs.thermal_3d(n=n, order=order)
            w.name = "frozen_3d"
            w.uth = 0.0
            if case == "imposed_fields":
                w.mass = 1e30
            parts = inputs.background(w)
            mem = TorchMemory()
            sim = Simulation(w, memory=mem, tuning=json.loads(args.tuning) if args.tuning else None)
            sim.load(parts)
            if case == "imposed_fields":
                z, y, x = np.meshgrid(*[np.arange(m, dtype=np.float64) for m in reversed(n)], indexing="ij")
                for c, name in enumerate(("Ex", "Ey", "Ez", "Bx", "By", "Bz")):
                    k = 2 * np.pi * (c + 1) / n[0]
                    f = 0.01 * (1.5 + np.cos(k * x + 0.3 * c) * np.cos(k * y) * np.cos(k * z + 0.7))
                    sim.set_field(name, f.astype(np.float32))
                del x, y, z
            sim.step(args.warmup)
            sim.sync()
            d0 = sim.diagnostics()
            clocks = Clocks(0)
            sim.profile_begin(args.steps)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(mem.stream)
            sim.step(args.steps)
            e1.record(mem.stream)
            torch.cuda.synchronize()
            phases, _ = sim.profile_end()
            clk = clocks.stop()
            d1 = sim.diagnostics()
            ms = e0.elapsed_time(e1) / args.steps
            sim.close()
            tun = json.loads(args.tuning) if args.tuning else None
            _, push_bytes, sp = algorithmic_bytes(
                w, parts.n, (d1["streamed"] - d0["streamed"]) / args.steps,
                (d1["live_tiles"] - d0["live_tiles"]) / args.steps * tile_cells(w, tun)
                if d1["live_tiles"] + d1["streamed"] > d0["live_tiles"] + d0["streamed"] else None)
            push_ms = phases["push"] / args.steps
            rows["%s_order%d" % (case, order)] = {
                "particle_steps_per_s": parts.n / (ms / 1e3), "ms_per_step": ms, "push_ms_per_step": push_ms,
                "push_zero_ms_per_step": phases["push_zero"] / args.steps,
                "sort_ms_per_step": phases["sort"] / args.steps, "sorts": d1["sorts"] - d0["sorts"],
                "streamed_fraction": (d1["streamed"] - d0["streamed"]) / (parts.n * args.steps),
                "push_roofline_frac": push_bytes / (push_ms / 1e3) / 1e9 / _peak(),
                "clocks": clk, "status": d1["status"]}
    for case in ("no_fields", "imposed_fields"):
        a, b = rows[case + "_order1"], rows[case + "_order2"]
        rows[case + "_quadratic_over_linear_time"] = b["ms_per_step"] / a["ms_per_step"]
        rows[case + "_quadratic_over_linear_push_time"] = b["push_ms_per_step"] / a["push_ms_per_step"]
    v = rows["no_fields_order2"]
    line = {"metric": METRIC, "value": v["particle_steps_per_s"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": v["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "frozen_3d: zero-temperature plasma %s cells, 8 ppc, periodic, orders 1 and 2, "
                                   "without fields and (immobile) in imposed fields (value: quadratic, no fields)"
                                   % "x".join(map(str, n)), "particles": int(np.prod(n)) * 8},
            "cases": rows, "paper_table2": TABLE2_FROZEN, "clocks": v["clocks"]}
    print(json.dumps(line), flush=True)
    if args.out:
        with open(args.out, "w") as f:
            f.write(json.dumps(line) + "\n")
    return 0


def _peak():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", 6800.0))
    except Exception:
        return 6800.0


def reference_arm(args):
    """The FP64 oracle timed on the host cores on the native arm's workload
    (a bounded crop; the whole run takes about a minute).  Under torchrun
    only rank 0 works."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w = workload(args.workload, args.scale, args.order)
    if args.workload in ("scan_2d", "adjoint_2d", "order_sweep", "frozen_3d"):
        print(json.dumps({"impl": "reference", "unavailable": "the oracle arm times the single-run workloads only"}))
        return 0
    cb = cpu_baseline(w, 45.0, steps=max(1, args.steps), warmup=args.warmup)
    n_full = w.n_particles_background()
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * n_full / cb["value"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(workload_config(w, n_full), timed="FP64 oracle on the host cores, a crop of the "
                                                             "workload; ms_per_step extrapolated to the full box"),
            "cpu_baseline": {"kind": cb["kind"], "cores": cb["cores"], "sample": cb["sample"], "value": cb["value"]},
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    if args.out:
        with open(args.out, "w") as f:
            f.write(json.dumps(line) + "\n")
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    if args.workload == "scan_2d":
        return scan_bench(args)
    if args.workload == "adjoint_2d":
        return adjoint_bench(args)
    if args.workload == "order_sweep":
        return order_sweep(args)
    if args.workload == "frozen_3d":
        return frozen_bench(args)
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    from paper_1310_0930_gb300.sim import Simulation, TorchMemory
    from paper_1310_0930_gb300 import inputs

    w = workload(args.workload, args.scale, args.order)
    tuning = json.loads(args.tuning) if args.tuning else None
    chunks = particle_chunks(w)
    n0 = sum(c.n for c in chunks)
    room = 4 * int(np.prod(w.n[:-1])) * w.ppc_total * 12 + 65536
    cap = n0 + room

    # ---- device-resident throughput (inputs already in HBM) ----------------
    mem = TorchMemory(device=local)
    sim = Simulation(w, tuning=tuning, capacity=cap, memory=mem)
    for c in chunks:
        sim.load(c)
    sim.step(args.warmup)
    sim.sync()
    d0 = sim.diagnostics()
    st = mem.stream
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = Clocks(local)
    sim.profile_begin(args.steps)
    barrier()
    torch.cuda.synchronize()
    ev0.record(st)
    sim.step(args.steps)
    ev1.record(st)
    torch.cuda.synchronize()
    barrier()
    phases, launches = sim.profile_end()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    d1 = sim.diagnostics()
    n_avg = 0.5 * (d0["n_particles"] + d1["n_particles"])
    ms, units = aggregate_replicas(ms, n_avg * args.steps)
    value = units / (ms / 1e3)
    streamed = (d1["streamed"] - d0["streamed"]) / args.steps
    live_cells = (d1["live_tiles"] - d0["live_tiles"]) / args.steps * tile_cells(w, tuning)
    step_bytes, push_bytes, sp = algorithmic_bytes(w, n_avg, streamed, live_cells if streamed > 0 else None)
    push_ms = phases["push"] / args.steps
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = push_bytes / (push_ms / 1e3) / 1e9
    # the particle phase's two kernels: zero-field tiles streamed
    # (ZERO_SLOT_BYTES per slot) and the staged tiles
    zero_ms = phases["push_zero"] / args.steps
    staged_ms = push_ms - zero_ms
    zero_bytes = streamed * ZERO_SLOT_BYTES
    staged_bytes = push_bytes - zero_bytes
    kernels = [
        {"kernel": "push_zero_kernel<%d,%d> (zero-field tiles)" % (w.dim, w.order), "slots_per_launch": streamed,
         "bytes_per_launch": zero_bytes, "avg_launch_ms": zero_ms,
         "achieved_gbs": zero_bytes / (zero_ms / 1e3) / 1e9 if zero_ms > 0 else None,
         "frac": zero_bytes / (zero_ms / 1e3) / 1e9 / peak if zero_ms > 0 else None},
        {"kernel": "tile classification + push_kernel<%d,%d> (live tiles)" % (w.dim, w.order),
         "particles_per_launch": n_avg - streamed, "bytes_per_launch": staged_bytes, "avg_launch_ms": staged_ms,
         "achieved_gbs": staged_bytes / (staged_ms / 1e3) / 1e9 if staged_ms > 0 else None,
         "frac": staged_bytes / (staged_ms / 1e3) / 1e9 / peak if staged_ms > 0 else None}]
    # the roofline reports the particle phase's dominant kernel by time
    dom = kernels[0] if zero_ms >= staged_ms else kernels[1]
    dom_bytes, dom_ms = dom["bytes_per_launch"], dom["avg_launch_ms"]
    units_dom = streamed if dom is kernels[0] else n_avg - streamed
    prof = None
    if not tuning:
        prof = (ZERO_PROFILE if dom is kernels[0] else STAGED_PROFILE).get((w.name, w.order))
    traffic = prof[0] * units_dom if prof else None
    issue = None
    if prof:
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        mhz = (clk or {}).get("sm_mhz") or 2070.0
        peak_issue = sms * 4 * mhz * 1e6  # four warp schedulers per SM, one instruction per clock each
        ach_issue = prof[1] * units_dom / (dom_ms / 1e3)
        issue = {"achieved": ach_issue, "peak": peak_issue, "unit": "warp-instructions/s",
                 "frac": ach_issue / peak_issue, "source": "profiles/" + prof[2]}
    status = d1["status"]
    sorts_timed = int(d1["sorts"] - d0["sorts"])
    sim.close()
    del sim

    # ---- the configured run from its first step to its last ----------------
    torch.cuda.empty_cache()
    full = None
    if world == 1 and not args.no_full_run and w.steps > args.steps:
        mem_f = TorchMemory(device=local)
        simf = Simulation(w, tuning=tuning, capacity=cap, memory=mem_f)
        for c in chunks:
            simf.load(c)
        simf.sync()
        f0 = simf.diagnostics()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        clocks_f = Clocks(local)
        torch.cuda.synchronize()
        e0.record(mem_f.stream)
        simf.step(w.steps)
        e1.record(mem_f.stream)
        torch.cuda.synchronize()
        clk_f = clocks_f.stop()
        ms_f = e0.elapsed_time(e1)
        f1 = simf.diagnostics()
        nf = 0.5 * (f0["n_particles"] + f1["n_particles"])
        sb_f, _, _ = algorithmic_bytes(w, nf, (f1["streamed"] - f0["streamed"]) / w.steps,
                                       (f1["live_tiles"] - f0["live_tiles"]) / w.steps * tile_cells(w, tuning)
                                       if f1["streamed"] > f0["streamed"] else None)
        full = {"value": nf * w.steps / (ms_f / 1e3), "ms_per_step": ms_f / w.steps, "steps": w.steps,
                "step_roofline_frac": sb_f / (ms_f / w.steps / 1e3) / 1e9 / peak, "clocks": clk_f,
                "sorts": int(f1["sorts"] - f0["sorts"]), "window_shifts": int(f1["shifts"]),
                "streamed_fraction": (f1["streamed"] - f0["streamed"]) / max(1.0, nf * w.steps),
                "status": f1["status"],
                "timed": "steps 1..%d from the loaded state, CUDA-graph replay, one pair of CUDA events" % w.steps}
        simf.close()
        del simf

    # ---- end to end through the C ABI with host buffers ----------------------
    e2e = None
    if not args.no_e2e:
        pinned = []
        h2d = 0
        for c in chunks:
            arrs = []
            for a in (c.cell, c.off, c.u, c.w):
                t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
                arrs.append(t)
                h2d += t.numel() * t.element_size()
            pinned.append(inputs.Particles(*[t.numpy() for t in arrs]))
        mem2 = TorchMemory(device=local)
        sim2 = Simulation(w, tuning=tuning, capacity=cap, memory=mem2)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for c in pinned:
            sim2.load(c)
        for _ in range(args.steps):
            sim2.step(1)
            sim2.sync()  # device -> host read of the step's status
        dd = sim2.diagnostics()  # energies and particle count back to the host
        t1 = time.perf_counter()
        barrier()
        sec, units_e2e = aggregate_replicas(t1 - t0, n0 * args.steps)
        e2e = {"value": units_e2e / sec, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d / args.steps), "d2h_bytes_per_step": int(96 + 96 / args.steps),
               "includes": "pic_load_particles from pinned host memory, %d x (pic_step + pic_sync), "
                           "pic_diagnostics (the handle, with its particle buffers of the configured "
                           "capacity, is created before the timed region)" % args.steps}
        sim2.close()
        del sim2, pinned

    # ---- the metric's other half: batched scan and adjoint against plain runs --
    # (memory the caching allocator kept from the runs above goes back first,
    # so that the adjoint finds the free memory it sizes its records by)
    torch.cuda.empty_cache()
    scan = adj = None
    if world == 1 and not args.no_scan:
        scan = scan_measure(args, args.scan_steps, 5, window_moves=True)
    if world == 1 and not args.no_adjoint:
        adj = adjoint_measure(args, args.adjoint_steps, 5)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, args.cpu_budget_s)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(workload_config(w, n0), particles_timed=int(n_avg),
                       sort_policy="fixed" if (tuning or {}).get("sort_policy") == 1 else "adaptive",
                       sorts_timed=sorts_timed,
                       steps_covered="steps %d..%d of the configured %d (after %d untimed warm-up steps)" % (
                           args.warmup + 1, args.warmup + args.steps, w.steps, args.warmup),
                       l2="inputs larger than L2 (%.1f GB particle state)" % (n_avg * sp / 1e9),
                       parallelism="replicas" if world > 1 else "single GPU",
                       timed="device-resident state, phase events recorded on the library stream"),
        "roofline": {"bound": "hbm", "achieved": dom_bytes / (dom_ms / 1e3) / 1e9 if dom_ms > 0 else None,
                     "peak": peak, "unit": "GB/s",
                     "frac": dom_bytes / (dom_ms / 1e3) / 1e9 / peak if dom_ms > 0 else None,
                     "traffic": traffic, "kernel": dom["kernel"],
                     "traffic_source": ("ncu capture of a scaled-down case of the same workload, %.1f B per %s "
                                        "scaled by the %ss of one launch, profiles/%s"
                                        % (prof[0], *(("slot", "slot") if dom is kernels[0] else
                                                      ("live-tile particle", "live-tile particle")), prof[2]))
                     if prof else None,
                     "issue": issue, "bytes_per_launch": dom_bytes, "avg_launch_ms": dom_ms,
                     "peak_source": "measured hbm_gbs (MEASURED_PEAKS.json)" if peaks else "fallback",
                     "phase": {"what": "particle phase: classification + push_kernel + push_zero_kernel",
                               "bytes_per_step": push_bytes, "ms_per_step": push_ms, "achieved": achieved,
                               "frac": achieved / peak},
                     "kernels": kernels},
        "step_roofline_frac": step_bytes / (ms / args.steps / 1e3) / 1e9 / peak,
        "phase_ms_per_step": {k: v / args.steps for k, v in phases.items()},
        "gpu_launches": int(launches),
        "clocks": clk,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "status": status,
        "full_run": full,
        "batched_scan": scan,
        "adjoint": adj,
    }
    if rank == 0:
        s = json.dumps(line)
        print(s, flush=True)
        if args.out:
            with open(args.out, "w") as f:
                f.write(s + "\n")
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

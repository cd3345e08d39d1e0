#!/usr/bin/env python3
"""Throughput benchmark of the fused finite-volume Euler step (cell updates/s).

Default workload: the 16.8M-triangle periodic unit square (4096 x 2048 quads,
seeded diagonals, nodes jittered 20 %), an isentropic vortex at Mach 0.5,
Hilbert cell order, FP32 state (plain float update; its error against the
FP64 path is reported), forward Euler at CFL 0.4.  Its state and geometry
(1.4 GB) are far larger than the L2, so every step streams from HBM: this is
the bandwidth headline.  One benchmark step = one call of the time loop (1,000
time steps, each one fused kernel, replayed as captured CUDA graphs) followed
by the FP64 conserved totals -- every row of the hot path.

Prints ONE JSON line.  Also reported: the same workload in FP64 (throughput,
speedup of FP32 over it, and the FP32 error against it) and with the
compensated FP32 update; the 1M-triangle channel with a circular-arc bump
(FP32 compensated, 10,000 time steps, and FP64); the roofline of the step
kernel; two steps per launch; normals from node coordinates; the 256-mesh
batch; the learned closure; the Mach 3 forward-facing step; the FP64 CPU
oracle timed on one host core; an end-to-end figure with host buffers.  The
key figures are repeated in a short `summary` object right after the scalars.
`--impl reference` times the CPU oracle alone.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1408_5715_gb300 import workloads as W  # noqa: E402

# Algorithmic bytes per cell update of one forward-Euler step: own state read
# and written once, 6 normal components + 1/V, 3 neighbour ids (neighbour
# states are counted as cache reuse, not DRAM traffic).
ALGO_BYTES = {"f32": 16 + 16 + 28 + 12, "f64": 32 + 32 + 56 + 12}
# The compensated FP32 update also reads and writes its 8-byte remainder.
COMP_BYTES = 8 + 8
FALLBACK_HBM_GBS = 6800.0
# The two-step launch (FP32, compensated) moves per tile cell and pair of
# updates: state in and out (32), geometry (32), tile-local neighbours (8),
# remainder in and out (16); halo reads are re-reads of other tiles' cells.
PAIR_BYTES = 32 + 32 + 8 + 16
# Normals from vertex coordinates (FP32): own state read and written, 3
# neighbour ids and 3 node ids, and the node coordinates (8 bytes per node,
# half a node per triangle) instead of 28 bytes of stored geometry.
VERTEX_BYTES = 16 + 16 + 12 + 12 + 4


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default="square_16m",
                   choices=["channel_bump_1m", "square_16m", "square_4m", "batch_256",
                            "vortex_square_small"])
    p.add_argument("--precision", default="f32", choices=["f32", "f64"])
    p.add_argument("--scheme", default="fe", choices=["fe", "rk2"])
    p.add_argument("--update", default=None, choices=["plain", "compensated"],
                   help="FP32 state update: plain float, or with the bfloat16 remainder "
                        "(default: the workload's)")
    p.add_argument("--order", default=None, choices=["identity", "shuffle", "rcm", "hilbert", "am1"])
    p.add_argument("--time-steps", type=int, default=None, help="time steps per benchmark step")
    p.add_argument("--no-extras", action="store_true", help="skip FP64 / 16M / CPU / e2e legs")
    p.add_argument("--blocking", type=int, default=1, choices=[1, 2],
                   help="time steps per kernel launch (2: tiles staged in shared memory, "
                        "dt evaluated once per pair)")
    p.add_argument("--tile", type=int, default=1024,
                   help="cells per tile: with --blocking 2 (512, 768, 1024 or 2048), or with "
                        "--variant 6 (32 .. 2048)")
    p.add_argument("--staged", action="store_true",
                   help="with --blocking 2: tile records by bulk copies (512 or 1024 cells)")
    p.add_argument("--closure", action="store_true",
                   help="step with the learned dissipation scale (untrained initial weights)")
    p.add_argument("--closure-engine", default="mma.sync", choices=["mma.sync", "tcgen05"],
                   help="tensor-core engine of the closure's MLP")
    p.add_argument("--variant", type=int, default=None,
                   help="force a step-kernel shape instead of autotuning")
    p.add_argument("--geometry", default="stored", choices=["stored", "vertex"],
                   help="stored normals, or normals formed from node coordinates on a grid")
    return p.parse_args()


WORKLOADS = {
    "channel_bump_1m": dict(make=W.channel_bump_1m, init="uniform", mach=0.5, time_steps=10000,
                            order="hilbert", update="compensated", desc="channel 3x1, 10% circular-arc bump, 1250x400 quads, "
                            "graded 4x, jitter 20%, far field M=0.5, slip walls"),
    "square_16m": dict(make=W.vortex_square_16m, init="vortex", mach=0.5, time_steps=1000,
                       order="hilbert", update="plain", desc="periodic unit square, 4096x2048 quads, jitter 20%, "
                       "isentropic vortex beta=5 M=0.5"),
    "square_4m": dict(make=lambda: W.periodic_square(2048, 1024, 4), init="vortex", mach=0.5,
                      time_steps=1000, order="hilbert", update="plain",
                      desc="periodic unit square, 2048x1024 quads, jitter 20%, isentropic "
                           "vortex beta=5 M=0.5 (a quarter of the 16.8M square, for profiles)"),
    "batch_256": dict(make=W.vortex_batch, batch=True, time_steps=1000, order="hilbert",
                      update="plain",
                      desc="256 periodic jittered squares, 4,900-200,704 triangles each "
                           "(log-uniform), vortex or uniform flow, Mach U(0.3, 0.8)"),
    "vortex_square_small": dict(make=W.vortex_square_small, init="vortex", mach=0.5,
                                time_steps=100, order="shuffle", update="compensated",
                                desc="periodic unit square, 64x32 quads, vortex"),
}


def initial_state(spec, mi):
    if spec["init"] == "uniform":
        return W.uniform_state(mi.n_tri, W.freestream(spec["mach"]))
    return W.isentropic_vortex(mi.centroids(), mach=spec["mach"])


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", FALLBACK_HBM_GBS)), "measured"
    return FALLBACK_HBM_GBS, "fallback"


KERNEL_SOURCES = ("kernels.h", "cell_math.cuh", "tile_math.cuh", "tma_util.cuh",
                  "launch_util.cuh", "kernels.cu", "tile_step.cu", "tma_step.cu", "pair_step.cu")


def kernel_source_hash():
    """Hash of the sources of the step kernels (ties a profile to the kernels
    it measured; any change to them makes the recorded traffic stale)."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1408_5715_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(name):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    h = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", txt)
    t = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    if not h or not t or h.group(1) != kernel_source_hash():
        return None
    return float(t.group(1))


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = os.path.join("/tmp", f"fv_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_id), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        rows = [[c.strip() for c in r] for r in rows if len(r) >= 8]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[0]) for r in rows if num(r[0]) is not None]
        mx = [num(r[1]) for r in rows if num(r[1]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if r[4 + j] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows),
                "power_w_max": max((num(r[2]) or 0.0) for r in rows)}


def gpu_smi_id():
    import torch
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    uuid = getattr(props, "uuid", None)
    if uuid is not None:
        s = str(uuid)
        return s if s.startswith("GPU-") else "GPU-" + s
    return os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0]


# ---------------------------------------------------------------------------
# our implementation
# ---------------------------------------------------------------------------
def make_mesh(B, spec, mi, precision, order):
    m = B.Mesh.from_input(mi, precision)
    prim = W.freestream(spec["mach"])
    m.set_freestream(*prim)
    perm = m.renumber(order, seed=1)
    return m, perm


def choose_variant(m, U, variant, scheme="fe"):
    """Autotunes the step-kernel shape (or forces one); returns a report."""
    if variant is not None:
        m.set_variant(variant)
        return {"variant": variant, "autotuned": False}
    best, us = m.autotune(U, scheme=scheme)
    return {"variant": best, "tile": m.tiling()[1] if best in (6, 7) else None, "autotuned": True,
            "us_per_step_by_variant": us}


def timed_loop(m, U, U0dev, time_steps, steps, warmup, scheme, cfl=0.4, flush=None,
               dist=None, closure=None):
    """Runs warmup + steps benchmark steps; returns per-step device times (s)."""
    import torch
    times = []
    for it in range(warmup + steps):
        U.copy_(U0dev)
        if flush is not None:
            flush.fill_(float(it))  # write > L2 so the step starts cold
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        m.step(U, time_steps, cfl, scheme=scheme, closure=closure, sync=False)
        m.totals(U)  # FP64 totals; synchronises
        e1.record()
        torch.cuda.synchronize()
        if it >= warmup:
            times.append(e0.elapsed_time(e1) / 1e3)
    m.status()  # raises if a bad state appeared
    return times


def run_ours(args):
    import torch
    import torch.distributed as tdist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        torch.cuda.set_device(local)
        tdist.init_process_group("nccl")
        dist = tdist
    else:
        torch.cuda.set_device(0)
    from paper_1408_5715_gb300 import binding as B
    from paper_1408_5715_gb300 import build as BLD
    if local == 0:
        BLD.build()
    if dist is not None:
        dist.barrier()
    B.load()

    spec = WORKLOADS[args.workload]
    if spec.get("batch"):
        return run_batch(args, B, spec, dist, world, rank)
    S = args.time_steps or spec["time_steps"]
    order = args.order or spec["order"]
    mi = spec["make"]()
    U0 = initial_state(spec, mi)
    n = mi.n_tri
    prec = args.precision
    tdt = torch.float32 if prec == "f32" else torch.float64
    m, perm = make_mesh(B, spec, mi, prec, order)
    update = (args.update or spec.get("update", "compensated")) if prec == "f32" else None
    if prec == "f32":
        m.set_compensation(update == "compensated")
    comp = update == "compensated"
    U0p = U0[perm]
    U0dev = torch.tensor(U0p, dtype=tdt, device="cuda")
    U = torch.empty_like(U0dev)
    closure = None
    if args.closure:
        if prec != "f32" or args.blocking != 1:
            raise SystemExit("--closure runs FP32, one step per launch")
        from paper_1408_5715_gb300 import closure_training as CT
        closure = B.Closure(CT.initial_theta(1, 0.3))
        m.set_closure_engine(args.closure_engine)
    if args.geometry == "vertex":
        if prec != "f32" or args.blocking != 1 or args.closure:
            raise SystemExit("--geometry vertex runs FP32, one step per launch, no closure")
        m.set_geometry("vertex")
    if args.blocking == 2:
        if prec != "f32" or args.scheme != "fe":
            raise SystemExit("--blocking 2 runs FP32 forward Euler")
        m.set_blocking(2, args.tile, args.staged)
        tune = {"blocking": 2, "tile": args.tile, "staged": args.staged}
    else:
        tune = choose_variant(m, U0dev, args.variant, args.scheme)
        if args.variant in (6, 7):
            m.set_blocking(1, args.tile)
            tune["tile"] = args.tile
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    with ClockSampler(gpu_smi_id()) as clk:
        times = timed_loop(m, U, U0dev, S, args.steps, args.warmup, args.scheme, flush=flush,
                           dist=dist, closure=closure)
    total = sum(times)
    if dist is not None:
        t = torch.tensor([total], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total = float(t.item())
    updates = n * S * args.steps * world
    value = updates / total
    stages = 2 if args.scheme == "rk2" else 1
    launches = S * stages // args.blocking
    avg_launch = total / (args.steps * launches)  # includes the per-call small kernels
    peak, peak_kind = measured_peaks()
    if args.blocking == 2:
        algo = kbytes = PAIR_BYTES if comp else PAIR_BYTES - COMP_BYTES
        kname = (f"{'k_step_pair_tma' if args.staged else 'k_step_pair'}"
                 f"<tile {args.tile}, {'compensated' if comp else 'plain'}>")
    else:
        algo = VERTEX_BYTES if args.geometry == "vertex" else ALGO_BYTES[prec]
        kbytes = algo + (COMP_BYTES if comp else 0)
        if args.closure:
            kfun = ("k_step_closure_tile" + ("_tc" if args.closure_engine == "tcgen05" else "")
                    if tune["variant"] == 7 else
                    "k_face_scales" + ("_tc" if args.closure_engine == "tcgen05" else "")
                    + " + k_step_scaled")
        else:
            kfun = {5: "k_step_tma", 6: "k_step_tile", 7: "k_step_tile_faces"}.get(
                tune["variant"], "k_step")
        kname = (f"{kfun}<{'float' if prec == 'f32' else 'double'}, "
                 f"{'RK2' if stages == 2 else 'FE'}, "
                 f"{'compensated' if comp else 'plain'}, shape {tune['variant']}"
                 f"{', vertex geometry' if args.geometry == 'vertex' else ''}>")
    achieved = algo * n / avg_launch / 1e9  # GB/s of one step-kernel launch
    U_final = U.double().cpu().numpy()
    e2e = e2e_leg(args, m, U0p, n, S, dist, closure)
    out = {
        "metric": "cell updates/s",
        "value": value,
        "unit": "cell-updates/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": prec,
        "data": "synthetic",
        "config": {"workload": args.workload, "mesh": spec["desc"], "cells": n,
                   "time_steps_per_step": S, "scheme": args.scheme, "cfl": 0.4, "order": order,
                   "update": update,
                   "geometry": ("normals from node coordinates on a grid of 2^%d" %
                                m.nodes()[1]) if args.geometry == "vertex" else "stored normals",
                   "dt": "CFL bound of the state at the start of each pair" if args.blocking == 2
                         else "CFL bound of the state at the start of each step",
                   "closure": f"learned dissipation scale, initial weights, MLP on "
                              f"{args.closure_engine}" if args.closure else None,
                   "parallelism": f"replicas{world}" if world > 1 else "single",
                   "kernel_shape": tune,
                   "l2": "256 MB written between steps (L2 flushed); state+geometry "
                         f"{n * (ALGO_BYTES[prec] + 8) / 1e6:.0f} MB"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": peak_kind,
                     "frac_of_nominal_7900": achieved / 7900.0,
                     "bytes_per_launch_per_cell": algo,
                     "kernel_bytes_per_launch_per_cell": kbytes,
                     "updates_per_launch": args.blocking,
                     "frac_with_kernel_bytes": kbytes * n / avg_launch / 1e9 / peak,
                     "kernel": kname,
                     "traffic": profiled_traffic(
                         f"step_pair_{args.workload}.md" if args.blocking == 2
                         else f"step_vertex_{args.workload}.md" if args.geometry == "vertex"
                         else f"step_{prec}{'' if comp or prec == 'f64' else '_plain'}"
                              f"_{args.workload}.md")},
        "e2e": e2e,
        "gpu_launches": args.steps * (launches + 4),
        "clocks": clk.summary(),
    }
    if rank == 0 and not args.no_extras and world == 1:
        extras(args, B, spec, mi, U0, U0p, perm, m, S, U_final, out)
        out["summary"] = summary(out)
        # the key figures right after the contract's scalars: the first
        # kilobyte of the line carries them
        head = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "summary")
        out = {**{k: out[k] for k in head if k in out},
               **{k: v for k, v in out.items() if k not in head}}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def run_batch(args, B, spec, dist, world, rank):
    """Many meshes of uneven size stepped together (one launch per time step
    for the whole batch): the same contract as the single-mesh line."""
    import torch
    if args.blocking != 1 or args.closure or args.scheme != "fe":
        raise SystemExit("the batch workload runs forward Euler, one step per launch")
    S = args.time_steps or spec["time_steps"]
    prec = args.precision
    tdt = torch.float32 if prec == "f32" else torch.float64
    items = spec["make"]()
    meshes, states = [], []
    for mi, prim, U0 in items:
        m = B.Mesh.from_input(mi, prec)
        m.set_freestream(*prim)
        perm = m.renumber(args.order or spec["order"], seed=1)
        meshes.append(m)
        states.append(U0[perm])
    batch = B.Batch(meshes)
    for m in meshes:
        m.close()
    if args.variant is not None:
        batch.set_variant(args.variant)
    update = (args.update or spec.get("update", "compensated")) if prec == "f32" else None
    if prec == "f32":
        batch.set_compensation(update == "compensated")
    host0 = batch.pack(states)
    flat0 = torch.tensor(host0, dtype=tdt, device="cuda")
    U = torch.empty_like(flat0)
    cells = int(sum(batch.sizes))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    times = []
    with ClockSampler(gpu_smi_id()) as clk:
        for it in range(args.warmup + args.steps):
            U.copy_(flat0)
            flush.fill_(float(it))
            torch.cuda.synchronize()
            if dist is not None:
                dist.barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            batch.step(U, S, 0.4, sync=False)
            batch.totals(U)
            e1.record()
            torch.cuda.synchronize()
            if it >= args.warmup:
                times.append(e0.elapsed_time(e1) / 1e3)
    batch.step(U, 0, 0.4)  # collects the error flag of the timed runs
    total = sum(times)
    if dist is not None:
        t = torch.tensor([total], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total = float(t.item())
    shape = batch.variant()
    avg_launch = total / (args.steps * S)
    peak, peak_kind = measured_peaks()
    kbytes = ALGO_BYTES[prec] + (COMP_BYTES if update == "compensated" else 0)
    achieved = ALGO_BYTES[prec] * cells / avg_launch / 1e9
    kname = {5: "k_step_tma", 6: "k_step_tile_batch", 0: "k_step_batch"}[shape]
    # end to end: the flat state in from pinned host memory and back, every step
    host_in = torch.tensor(host0, dtype=tdt).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    te = []
    for it in range(2):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        U.copy_(host_in, non_blocking=True)
        batch.step(U, S, 0.4, sync=False)
        tot = batch.totals(U)
        host_out.copy_(U, non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        if it > 0:
            te.append(e0.elapsed_time(e1) / 1e3)
    assert np.isfinite(tot).all()
    nb = host_in.numel() * host_in.element_size()
    out = {
        "metric": "cell updates/s", "value": cells * S * args.steps * world / total,
        "unit": "cell-updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": prec, "data": "synthetic",
        "config": {"workload": args.workload, "mesh": spec["desc"], "cells": cells,
                   "padded_cells": batch.n_padded, "meshes": batch.n_meshes,
                   "time_steps_per_step": S, "scheme": "fe", "cfl": 0.4,
                   "order": args.order or spec["order"], "update": update,
                   "dt": "per mesh: CFL bound of its state at the start of each step",
                   "parallelism": f"replicas{world}" if world > 1 else "single",
                   "kernel_shape": {"variant": shape, "autotuned": False},
                   "l2": "256 MB written between steps (L2 flushed); state+geometry "
                         f"{cells * (ALGO_BYTES[prec] + 8) / 1e6:.0f} MB"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": peak_kind,
                     "frac_of_nominal_7900": achieved / 7900.0,
                     "bytes_per_launch_per_cell": ALGO_BYTES[prec],
                     "kernel_bytes_per_launch_per_cell": kbytes, "updates_per_launch": 1,
                     "frac_with_kernel_bytes": kbytes * cells / avg_launch / 1e9 / peak,
                     "kernel": f"{kname}<{'float' if prec == 'f32' else 'double'}, FE, "
                               f"{update or 'plain'}>",
                     "traffic": profiled_traffic(
                         f"step_{prec}{'_plain' if update == 'plain' else ''}_{args.workload}.md")},
        "e2e": {"value": cells * S / statistics.mean(te), "unit": "cell-updates/s",
                "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb + 32 * batch.n_meshes,
                "api": "fv_batch_step + fv_batch_totals on host-copied state"},
        "gpu_launches": args.steps * (S + 4),
        "clocks": clk.summary(),
    }
    batch.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def e2e_leg(args, m, U0p, n, S, dist=None, closure=None):
    """The same metric end to end through the public API: every step copies
    the state in from pinned host memory, steps, reads the totals and copies
    the state back."""
    import torch
    tdt = torch.float32 if args.precision == "f32" else torch.float64
    host_in = torch.tensor(U0p, dtype=tdt).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    Ud = torch.empty(host_in.shape, dtype=tdt, device="cuda")
    times = []
    for it in range(2):
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        Ud.copy_(host_in, non_blocking=True)
        m.step(Ud, S, 0.4, scheme=args.scheme, closure=closure, sync=False)
        tot = m.totals(Ud)
        host_out.copy_(Ud, non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        if it > 0:
            times.append(e0.elapsed_time(e1) / 1e3)
    assert np.isfinite(tot).all()
    t = statistics.mean(times)
    world = 1
    if dist is not None:
        world = dist.get_world_size()
        tt = torch.tensor([t], device="cuda", dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    nb = host_in.numel() * host_in.element_size()
    return {"value": world * n * S / t, "unit": "cell-updates/s",
            "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb + 32,
            "api": "fv_step + fv_conserved_totals on host-copied state"}


def mesh_run(B, spec, mi, U0, prec, update, time_steps, steps=2, warmup=1):
    """One single-mesh workload in one precision and update: autotuned shape,
    timed like the main line (L2 flushed between benchmark steps).  Returns
    the report and the final state in the mesh's input cell order."""
    import torch
    m, perm = make_mesh(B, spec, mi, prec, spec["order"])
    comp = prec == "f32" and update == "compensated"
    if prec == "f32":
        m.set_compensation(comp)
    tdt = torch.float32 if prec == "f32" else torch.float64
    U0d = torch.tensor(U0[perm], dtype=tdt, device="cuda")
    U = torch.empty_like(U0d)
    tune = choose_variant(m, U0d, None)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    tt = timed_loop(m, U, U0d, time_steps, steps, warmup, "fe", flush=flush)
    v = mi.n_tri * time_steps / statistics.mean(tt)
    peak, _ = measured_peaks()
    gbs = ALGO_BYTES[prec] * v / 1e9
    res = {"value": v, "unit": "cell-updates/s", "dtype": prec, "cells": mi.n_tri,
           "time_steps": time_steps, "order": spec["order"], "kernel_shape": tune,
           "achieved_gbs": gbs, "frac_of_measured_hbm": gbs / peak,
           "frac_with_kernel_bytes": (ALGO_BYTES[prec] + (COMP_BYTES if comp else 0)) * v / 1e9
                                     / peak}
    if prec == "f32":
        res["update"] = update
    final = np.empty(U0.shape)
    final[perm] = U.double().cpu().numpy()
    del U, U0d, flush
    m.close()
    return res, final


def rel_l2_rho(a, b):
    return float(np.linalg.norm(a[:, 0] - b[:, 0]) / np.linalg.norm(b[:, 0]))


def extras(args, B, spec, mi, U0, U0p, perm, m32, S, U32_final, out):
    n = mi.n_tri
    cfg = out["config"]
    if args.precision == "f32" and args.blocking == 1 and args.geometry == "stored" \
            and not args.closure:
        # ---- same workload in FP64: throughput, speedup, error of FP32 against it
        r64, U64 = mesh_run(B, spec, mi, U0, "f64", None, S, steps=1, warmup=1)
        main32 = np.empty(U0.shape)
        main32[perm] = U32_final
        r64["speedup_fp32_over_fp64"] = out["value"] / r64["value"]
        r64["fp32_rel_l2_rho_vs_fp64"] = rel_l2_rho(main32, U64)
        r64["tolerance"] = 1e-5
        out["fp64"] = r64
        # ---- the other FP32 update on the same workload
        other = "plain" if cfg["update"] == "compensated" else "compensated"
        r, U = mesh_run(B, spec, mi, U0, "f32", other, S)
        r["rel_l2_rho_vs_fp64"] = rel_l2_rho(U, U64)
        out[f"fp32_{other}"] = r
        del U64, U
    # ---- the other single-mesh workload: the 1M channel (L2-sized,
    # 10,000 steps, compensated update) or the 16.8M square (the HBM headline)
    name = "channel_bump_1m" if args.workload != "channel_bump_1m" else "square_16m"
    spec2 = WORKLOADS[name]
    mi2 = spec2["make"]()
    U02 = initial_state(spec2, mi2)
    res = {"cells": mi2.n_tri, "order": spec2["order"], "mesh": spec2["desc"]}
    res["f32"], U32 = mesh_run(B, spec2, mi2, U02, "f32", spec2["update"], spec2["time_steps"])
    res["f32"]["traffic"] = profiled_traffic(
        f"step_f32{'' if spec2['update'] == 'compensated' else '_plain'}_{name}.md")
    res["f64"], U64 = mesh_run(B, spec2, mi2, U02, "f64", None, spec2["time_steps"], steps=1)
    res["speedup_fp32_over_fp64"] = res["f32"]["value"] / res["f64"]["value"]
    res["fp32_rel_l2_rho_vs_fp64"] = rel_l2_rho(U32, U64)
    res["tolerance"] = 1e-5
    out[name] = res
    del U32, U64
    # a leg that fails reports its error; the headline line is still printed
    def leg(name, fn):
        try:
            out[name] = fn(B)
        except Exception as e:  # noqa: BLE001
            out[name] = {"error": f"{type(e).__name__}: {e}"}
    # ---- the same loop with each step launched only after the previous one
    if args.precision == "f32" and args.blocking == 1:
        leg("unchained", lambda B_: unchained_leg(m32, U0p, S, args.scheme, out["value"]))
    # ---- normals from node coordinates against stored normals
    leg("vertex_geometry", vertex_leg)
    # ---- two steps per launch (temporal blocking) on the same workloads
    leg("pairs", pair_leg)
    # ---- many meshes in one launch per step (256 periodic squares, 5k-200k cells)
    leg("batched", batched_leg)
    # ---- learned dissipation scale: cost per step on the 250k-cell coarse channel
    leg("learned", learned_leg)
    # ---- the paper's own case: Mach 3 forward-facing step to t = 4
    leg("forward_step", forward_step_leg)
    # ---- FP64 CPU oracle on one host core, bounded sample of this workload
    out["cpu_baseline"] = cpu_baseline(spec, mi, U0, budget_s=12.0)


def summary(out):
    """The key figures of the line in a few hundred bytes (placed right after
    the contract's scalar keys)."""
    def g(d, *path):
        for p in path:
            if not isinstance(d, dict) or p not in d:
                return None
            d = d[p]
        return d

    def r3(x):
        return None if x is None else float(f"{x:.4g}")
    other = "channel_bump_1m" if out["config"]["workload"] != "channel_bump_1m" else "square_16m"
    return {
        "workload": out["config"]["workload"],
        "value": r3(out["value"]), "roofline_frac": r3(out["roofline"]["frac"]),
        "traffic_per_launch": out["roofline"]["traffic"],
        "fp64_value": r3(g(out, "fp64", "value")),
        "fp32_speedup_over_fp64": r3(g(out, "fp64", "speedup_fp32_over_fp64")),
        "fp32_rel_l2_rho_vs_fp64": r3(g(out, "fp64", "fp32_rel_l2_rho_vs_fp64")),
        "compensated_value": r3(g(out, "fp32_compensated", "value")),
        other: {"f32": r3(g(out, other, "f32", "value")),
                "f32_frac": r3(g(out, other, "f32", "frac_of_measured_hbm")),
                "f64": r3(g(out, other, "f64", "value")),
                "fp32_rel_l2_rho_vs_fp64": r3(g(out, other, "fp32_rel_l2_rho_vs_fp64"))},
        "batched": r3(g(out, "batched", "value")),
        "batched_frac_72B": r3(g(out, "batched", "frac_of_measured_hbm_72B")),
        "pairs_speedup_16m": r3(g(out, "pairs", "square_16m", "speedup_over_single_step")),
        "learned_overhead": r3(g(out, "learned", "overhead")),
        "cpu_baseline": r3(g(out, "cpu_baseline", "value")),
        "e2e": r3(out["e2e"]["value"]),
        "peak_gbs": out["roofline"]["peak"],
    }


def unchained_leg(m, U0p, S, scheme, chained_value):
    """The main loop without programmatic dependent launch (each step kernel
    waits for the previous one to finish before it is scheduled)."""
    import torch
    U0d = torch.tensor(U0p, dtype=torch.float32, device="cuda")
    U = torch.empty_like(U0d)
    m.set_launch_chaining(False)
    try:
        tt = timed_loop(m, U, U0d, S, 2, 1, scheme)
    finally:
        m.set_launch_chaining(True)
    v = U0p.shape[0] * S / statistics.mean(tt)
    return {"value": v, "unit": "cell-updates/s", "chained_over_unchained": chained_value / v}


def vertex_leg(B, time_steps=1000):
    """Normals formed from node coordinates (Sec. 7's alternative to stored
    normals) against stored normals: FP32 compensated, Hilbert order,
    autotuned shape, CFL 0.4.  The vertex form runs on the nodes snapped to
    its grid; the density difference between the two runs measures what the
    snapping moves (the vertex form is bitwise the stored records of the
    snapped mesh, checked by the tests)."""
    import torch
    peak, _ = measured_peaks()
    res = {}
    for name in ("channel_bump_1m", "square_16m"):
        spec = WORKLOADS[name]
        mi = spec["make"]()
        U0 = initial_state(spec, mi)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        r = {"cells": mi.n_tri, "order": "hilbert", "time_steps": time_steps}
        finals = {}
        for geom in ("stored", "vertex"):
            m, perm = make_mesh(B, spec, mi, "f32", "hilbert")
            if geom == "vertex":
                m.set_geometry("vertex")
                r["grid_exponent"] = m.nodes()[1]
            U0d = torch.tensor(U0[perm], dtype=torch.float32, device="cuda")
            U = torch.empty_like(U0d)
            tune = choose_variant(m, U0d, None)
            tt = timed_loop(m, U, U0d, time_steps, 3, 2, "fe", flush=flush)
            v = mi.n_tri * time_steps / statistics.median(tt)
            algo = VERTEX_BYTES if geom == "vertex" else ALGO_BYTES["f32"]
            gbs = algo * v / 1e9
            r[geom] = {"value": v, "unit": "cell-updates/s", "kernel_shape": tune,
                       "bytes_per_update": algo, "achieved_gbs": gbs,
                       "frac_of_measured_hbm": gbs / peak,
                       "traffic": profiled_traffic(f"step_vertex_{name}.md" if geom == "vertex"
                                                   else f"step_f32_{name}.md")}
            out = np.empty(U0.shape)
            out[perm] = U.double().cpu().numpy()
            finals[geom] = out
            del U, U0d
            m.close()
        r["speedup_vertex_over_stored"] = r["vertex"]["value"] / r["stored"]["value"]
        a, b = finals["vertex"][:, 0], finals["stored"][:, 0]
        r["rel_l2_rho_vertex_vs_stored"] = float(np.linalg.norm(a - b) / np.linalg.norm(b))
        res[name] = r
        del flush
    return res


def pair_leg(B, time_steps=1000):
    """Two forward-Euler steps per launch on shared-memory tiles (Hilbert order),
    against one launch per step on the same mesh; FP32 with the workload's
    update (plain on the square, compensated on the channel), CFL 0.4 (one dt
    per pair for the two-step launch)."""
    import torch
    peak, _ = measured_peaks()
    res = {}
    for name in ("channel_bump_1m", "square_16m"):
        spec = WORKLOADS[name]
        mi = spec["make"]()
        U0 = initial_state(spec, mi)
        m, perm = make_mesh(B, spec, mi, "f32", "hilbert")
        comp = spec["update"] == "compensated"
        m.set_compensation(comp)
        pair_bytes = PAIR_BYTES if comp else PAIR_BYTES - COMP_BYTES
        U0d = torch.tensor(U0[perm], dtype=torch.float32, device="cuda")
        U = torch.empty_like(U0d)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        single = choose_variant(m, U0d, None)
        ts = timed_loop(m, U, U0d, time_steps, 2, 1, "fe", flush=flush)
        v1 = mi.n_tri * time_steps / statistics.mean(ts)
        by_tile = {}
        for tile, staged in ((512, False), (768, False), (1024, False), (2048, False),
                             (512, True), (1024, True)):
            m.set_blocking(2, tile, staged)
            tt = timed_loop(m, U, U0d, time_steps, 2, 1, "fe", flush=flush)
            by_tile[f"{tile}{'-staged' if staged else ''}"] = (
                mi.n_tri * time_steps / statistics.mean(tt))
        best = max(by_tile, key=by_tile.get)
        v2 = by_tile[best]
        launch = 2 * mi.n_tri / v2  # seconds per two-step launch (per-call kernels included)
        gbs = pair_bytes * mi.n_tri / launch / 1e9
        res[name] = {"cells": mi.n_tri, "order": "hilbert", "time_steps": time_steps,
                     "single_step": {"value": v1, "kernel_shape": single},
                     "value": v2, "unit": "cell-updates/s", "tile": best,
                     "value_by_tile": by_tile, "speedup_over_single_step": v2 / v1,
                     "achieved_gbs": gbs, "frac_of_measured_hbm": gbs / peak,
                     "update": spec["update"],
                     "single_step_equivalent_gbs":
                         (ALGO_BYTES["f32"] + (COMP_BYTES if comp else 0)) * v2 / 1e9,
                     "kernel": (f"k_step_pair_tma<tile {best.split('-')[0]}, {spec['update']}>"
                                if best.endswith("staged")
                                else f"k_step_pair<tile {best}, {spec['update']}>")}
        del U, U0d, flush
        m.close()
    return res


def batched_leg(B, time_steps=1000):
    """256 meshes in one launch per step, every kernel shape, with the plain and
    the compensated FP32 update; FP32 error of each against the FP64 path on
    the smallest and the largest mesh."""
    import torch
    items = W.vortex_batch()
    meshes, states = [], []
    for mi, prim, U0 in items:
        m = B.Mesh.from_input(mi, "f32")
        m.set_freestream(*prim)
        perm = m.renumber("hilbert")
        meshes.append(m)
        states.append(U0[perm])
    batch = B.Batch(meshes)
    for m in meshes:
        m.close()
    flat0 = torch.tensor(batch.pack(states), dtype=torch.float32, device="cuda")
    U = torch.empty_like(flat0)
    cells = int(sum(batch.sizes))
    peak, _ = measured_peaks()
    # error samples: the smallest and the largest mesh that start from a
    # vortex (a uniform stream stays uniform and tests nothing)
    vortex = [k for k, (_, _, U0) in enumerate(items) if np.ptp(U0[:, 0]) > 0]
    sizes = np.asarray(batch.sizes)
    sample = (min(vortex, key=lambda k: sizes[k]), max(vortex, key=lambda k: sizes[k]))
    ref64 = {}
    for k in sample:
        mi, prim, U0 = items[k]
        m64 = B.Mesh.from_input(mi, "f64")
        m64.set_freestream(*prim)
        perm = m64.renumber("hilbert")
        U64 = torch.tensor(U0[perm], dtype=torch.float64, device="cuda")
        m64.step(U64, time_steps, 0.4)
        ref64[k] = U64[:, 0].cpu().numpy()
        m64.close()
    res = {"meshes": batch.n_meshes, "cells": cells, "padded_cells": batch.n_padded,
           "time_steps": time_steps, "dtype": "f32", "order": "hilbert", "tolerance": 1e-5,
           "launches_per_step": time_steps + 4}
    for update in ("plain", "compensated"):
        batch.set_compensation(update == "compensated")
        by_shape = {}
        for shape in (5, 6, 0):
            batch.set_variant(shape)
            times = []
            for it in range(3):
                U.copy_(flat0)
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                batch.step(U, time_steps, 0.4, sync=False)
                batch.totals(U)
                e1.record()
                torch.cuda.synchronize()
                if it > 0:
                    times.append(e0.elapsed_time(e1) / 1e3)
            batch.step(U, 0, 0.4)  # collects the error flag of the runs above
            by_shape[shape] = statistics.mean(times)
            if shape == 0:
                got = batch.unpack(U.cpu().numpy())
        best = min(by_shape, key=by_shape.get)
        v = cells * time_steps / by_shape[best]
        kb = ALGO_BYTES["f32"] + (COMP_BYTES if update == "compensated" else 0)
        errs = {f"mesh_{k}_{items[k][0].n_tri}_cells":
                float(np.linalg.norm(got[k][:, 0] - ref64[k]) / np.linalg.norm(ref64[k]))
                for k in sample}
        res[update] = {
            "value": v, "unit": "cell-updates/s", "shape": best,
            "kernel": {5: "k_step_tma<float, FE, {u}, batch>",
                       6: "k_step_tile_batch<float, FE, {u}>",
                       0: "k_step_batch<float, FE, {u}>"}[best].format(u=update),
            "value_by_shape": {k: cells * time_steps / t for k, t in by_shape.items()},
            "fp32_rel_l2_rho_vs_fp64": errs,
            "frac_of_measured_hbm_72B": ALGO_BYTES["f32"] * v / 1e9 / peak,
            "frac_with_kernel_bytes": kb * v / 1e9 / peak}
    # the headline of the leg: the plain float update, whose error is reported
    res.update({k: res["plain"][k] for k in ("value", "unit", "shape", "kernel")})
    res["frac_of_measured_hbm_72B"] = res["plain"]["frac_of_measured_hbm_72B"]
    batch.close()
    return res


def forward_step_leg(B, t_end=4.0):
    """Mach 3 over a forward-facing step (Sec. 7.1), FP32, CFL 0.4: wall time to
    simulate t_end on the 65,664-triangle mesh of the family (refined 12.5x
    toward the corner), how far the 410,400-triangle mesh (the paper's
    largest size) gets before the corner expansion drives a pressure
    non-positive, and that mesh to t_end with the maximum wave speed."""
    import torch
    prim = W.mach3_inflow()

    def run(mi, t_end, timed, wave="average"):
        m = B.Mesh.from_input(mi, "f32")
        m.set_freestream(*prim)
        m.set_wave_speed(wave)
        perm = m.renumber("hilbert")
        U0 = torch.tensor(W.uniform_state(mi.n_tri, prim)[perm], dtype=torch.float32,
                          device="cuda")
        U = U0.clone()
        tune = None
        if timed:
            tune = choose_variant(m, U0, None)
            m.step(U, 200, 0.4)  # warm-up (graph capture)
            U.copy_(U0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        t, steps, failed = 0.0, 0, None
        while t < t_end - 1e-12:
            chunk = min(0.1, t_end - t)
            dt = m.compute_dt(U, 0.4)
            n = int(math.ceil(chunk / (0.9 * dt))) + 2
            try:
                t += m.step(U, n, 0.4, t_stop=chunk)
            except B.FVError as e:
                failed = f"non-positive state between t = {t:.2f} and {t + chunk:.2f} ({e})"
                break
            steps += n
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        rho = U[:, 0].double()
        res = {"cells": mi.n_tri, "t_reached": t, "steps_launched": steps, "wall_s": wall,
               "order": "hilbert", "kernel_shape": tune}
        if failed:
            res["failed"] = failed
        else:
            res.update({"value": mi.n_tri * steps / wall, "unit": "cell-updates/s",
                        "rho_max_over_inflow": float(rho.max()) / prim[0],
                        "rho_min_over_inflow": float(rho.min()) / prim[0]})
        m.close()
        return res

    out = run(W.forward_step_65k(), t_end, True)
    out["dtype"] = "f32"
    out["paper_size_mesh"] = run(W.forward_step_394k(), t_end, False)
    # the same mesh with the one-sided maximum wave speed (Rusanov reading)
    out["paper_size_mesh_max_wave"] = run(W.forward_step_394k(), t_end, True, "max")
    return out


def learned_leg(B, time_steps=2000):
    import torch
    from paper_1408_5715_gb300 import closure_training as CT
    mi = W.channel_bump(625, 200, seed=5)
    m = B.Mesh.from_input(mi, "f32")
    m.set_freestream(*W.freestream(0.5))
    m.renumber("hilbert")
    cl = B.Closure(CT.initial_theta(1, 0.3))
    U0 = torch.tensor(W.uniform_state(mi.n_tri, W.freestream(0.5)), dtype=torch.float32,
                      device="cuda")
    plain_shape = choose_variant(m, U0, None)  # the plain step in its fastest shape
    cost = CT.step_cost(m, cl, steps=time_steps)
    # the learned step on shape 7's tiles (one kernel per step), by tile size
    keep_variant, keep_tile = m.tiling()
    by_tile = {}
    m.set_variant(7)
    # the standard sizes and those that fill one or two waves of two blocks per SM
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    fit = [-(-mi.n_tri // (w * 2 * sms)) for w in (1, 2)]
    for tile in sorted({256, 512, 1024} | {(t + 31) // 32 * 32 for t in fit if 64 <= t <= 1024}):
        m.set_blocking(1, tile)
        by_tile[tile] = CT.step_cost(m, cl, steps=time_steps)["learned"]
    best_tile = min(by_tile, key=by_tile.get)
    # the same two forms with the MLP on tcgen05 (128-row MMAs into tensor memory)
    m.set_closure_engine("tcgen05")
    m.set_blocking(1, best_tile)
    tc = {"tile_%d" % best_tile: CT.step_cost(m, cl, steps=time_steps)["learned"]}
    m.set_variant(keep_variant)
    m.set_blocking(1, keep_tile)
    tc["two_passes"] = CT.step_cost(m, cl, steps=time_steps)["learned"]
    m.set_closure_engine("mma.sync")
    learned_us = min(cost["learned"], by_tile[best_tile])
    n = mi.n_tri
    nbr, _, _ = m.export()
    # tensor-core work per MLP row: layer 1 (K = 16: 8 features, 3 bias rows,
    # padding) and layer 2 (K = 32, and a K = 16 slice for its bias rows)
    mma_flops = 2 * (16 * 32 + 48 * 32)
    # MLP rows per step: each face once
    rows = int((nbr < 0).sum() + (nbr >= 0).sum() // 2)
    res = {"cells": n, "order": "hilbert", "time_steps": time_steps,
           "us_per_step_plain": cost["plain"], "plain_kernel_shape": plain_shape,
           "us_per_step_learned_two_passes": cost["learned"],
           "us_per_step_learned_tiles": by_tile,
           "us_per_step_learned": learned_us,
           "us_per_step_learned_tcgen05": tc,
           "value": n / (learned_us * 1e-6), "unit": "cell-updates/s",
           "overhead": learned_us / cost["plain"],
           "mlp_rows_per_cell": rows / n,
           "mma_flops_per_cell": mma_flops * rows / n,
           "mma_tflops": mma_flops * rows / (learned_us * 1e-6) / 1e12,
           "kernel": (f"k_step_closure_tile<FE, compensated, tile {best_tile}>"
                      if by_tile[best_tile] < cost["learned"]
                      else "k_face_scales + k_step_scaled<FE, compensated>")
                     + " (mma.sync m16n8k16 bf16)"}
    m.close()
    cl.close()
    return res


def cpu_baseline(spec, mi, U0, budget_s=12.0):
    import oracle
    oracle.build()
    uinf = W.conserved(*W.freestream(spec["mach"]))
    om = oracle.Mesh(mi.xy, mi.tri, mi.canon, mi.bnd, mi.default_bc, uinf)
    t0 = time.perf_counter()
    om.run(U0, 1, 0.4)
    one = time.perf_counter() - t0
    nsteps = max(1, int(budget_s / max(one, 1e-6)))
    t0 = time.perf_counter()
    _, _, done, _ = om.run(U0, nsteps, 0.4)
    el = time.perf_counter() - t0
    return {"value": mi.n_tri * done / el, "unit": "cell-updates/s", "cores": 1, "kind": "oracle",
            "sample": f"{done} forward-Euler steps of the full {mi.n_tri}-cell mesh, FP64, "
                      f"single thread ({el:.1f} s)",
            "cpu": cpu_model()}


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return os.uname().machine


# ---------------------------------------------------------------------------
# reference arm: the FP64 oracle as it stands, on the host cores
# ---------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    spec = WORKLOADS[args.workload]
    if spec.get("batch"):
        # a bounded sample of the batch: its largest mesh (every mesh of the
        # batch is stepped the same way, one after another on the CPU)
        items = spec["make"]()
        mi, prim, U0 = max(items, key=lambda it: it[0].n_tri)
        uinf = W.conserved(*prim)
    else:
        mi = spec["make"]()
        U0 = initial_state(spec, mi)
        uinf = W.conserved(*W.freestream(spec["mach"]))
    om = oracle.Mesh(mi.xy, mi.tri, mi.canon, mi.bnd, mi.default_bc, uinf)
    # time steps per benchmark step: a bounded sample of the workload (one
    # step of the 16.8M-cell square takes a few seconds on one core)
    per_step = 1 if mi.n_tri > 4_000_000 else 2
    for _ in range(args.warmup):
        om.run(U0, 1, 0.4)
    t0 = time.perf_counter()
    done = 0
    for _ in range(args.steps):
        _, _, d, _ = om.run(U0, per_step, 0.4)
        done += d
    el = time.perf_counter() - t0
    v = mi.n_tri * done / el
    out = {"metric": "cell updates/s", "value": v, "unit": "cell-updates/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "impl": "reference",
           "config": {"workload": args.workload, "mesh": spec["desc"], "cells": mi.n_tri,
                      "time_steps_per_step": per_step, "scheme": "fe", "cfl": 0.4},
           "cpu_baseline": {"value": v, "unit": "cell-updates/s", "cores": 1, "kind": "oracle",
                            "sample": f"{per_step} FP64 forward-Euler steps of the full mesh "
                                      f"({mi.n_tri} cells) per benchmark step, single thread",
                            "cpu": cpu_model()},
           "e2e": {"value": v, "unit": "cell-updates/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse_args()
    if args.warmup < 0 or args.steps < 1:
        raise SystemExit("need --steps >= 1")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

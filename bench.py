#!/usr/bin/env python
"""Benchmark of the hot path: one step = pi_bin + pi_interact (cell index,
histogram, scan, stable scatter, cutoff interaction) on the 2,097,152-particle
uniform workload (64^3 cells, r_c = 1/64, ~8 particles per cell, Gaussian
kernel with h = r_c/2), inputs resident in HBM, through the C ABI.

Prints one JSON line.  ``value`` is within-cutoff (ordered) pair interactions
per second over the full step, summed over ranks; ``e2e`` is the same metric
through ``pi_run_host`` with host buffers and the copies inside the timed
region; ``roofline`` covers the interaction kernel (FP32 ALU bound);
``cpu_baseline`` times the FP64 CPU oracle on this host.

``--impl reference`` times the oracle instead (the reference arm of this
build: there is no reference implementation to run).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU: torchrun ... bench.py --gpus N: independent replicas, one per GPU.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2406_16091_gb300 import workloads as W  # noqa: E402

METRIC = "within-cutoff pair interactions/s"
UNIT = "pairs/s"
# FLOP per within-cutoff ordered pair in the per-target formulation:
# 3 (displacement) + 5 (r^2) + 1 (scale) + 1 (exp2) + 1 (S) + 6 (V)
FLOP_PER_PAIR = 17
FP32_LANES_PER_SM = 128


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3000)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default="scale", choices=sorted(W.WORKLOADS))
    p.add_argument("--algo", choices=["tiled", "ppnl"], default="tiled")
    p.add_argument("--precision", choices=["fp32", "kahan"], default="fp32")
    p.add_argument("--e2e-steps", type=int, default=100)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--flush-mb", type=int, default=512)
    return p.parse_args()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            return d, "measured"
        except Exception:
            pass
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def source_hash(paths):
    h = hashlib.sha256()
    for p in paths:
        h.update(open(p, "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel_key, src_hash):
    """Per-launch DRAM bytes from the committed ncu summary, if it was taken
    on the current source of the kernel."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path)).get(kernel_key)
    except Exception:
        return None
    if not d or d.get("source_hash") != src_hash:
        return None
    return d


class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id):
        self.proc = None
        self.bus_id = bus_id

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "50"]
        if self.bus_id:
            cmd.insert(1, f"--id={self.bus_id}")
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.15)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.1)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------- reference arm


def oracle_step_sample(w: W.Workload, x, y, z, layers: int):
    """The workload's particles in the slab z < layers cells (same density and
    per-cell occupancy), binned and interacted by the oracle."""
    import oracle

    zc = layers / w.cells_per_axis() * (w.hi[2] - w.lo[2]) + w.lo[2]
    sel = z < np.float32(zc)
    xs, ys, zs = x[sel], y[sel], z[sel]
    hi = (w.hi[0], w.hi[1], zc)
    t0 = time.perf_counter()
    b = oracle.bin_particles(xs, ys, zs, w.lo, hi, w.rc)
    r = oracle.interact(b, w.rc, w.h)
    dt = time.perf_counter() - t0
    return int(r.nbr.sum()), dt, len(xs)


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle

    oracle.build()
    w = W.WORKLOADS[args.workload]
    x, y, z = w.positions()
    ncell = w.cells_per_axis()
    # size each step's slab so that warm-up + timed steps take about 90 s
    _, dt1, _ = oracle_step_sample(w, x, y, z, 1)
    per_step = 90.0 / max(1, args.steps + args.warmup)
    layers = int(max(1, min(ncell, per_step / max(dt1, 1e-6))))
    for _ in range(args.warmup):
        oracle_step_sample(w, x, y, z, layers)
    pairs_total, t_total, nparts = 0, 0.0, 0
    for _ in range(args.steps):
        p, dt, nparts = oracle_step_sample(w, x, y, z, layers)
        pairs_total += p
        t_total += dt
    value = pairs_total / t_total
    cores = oracle.num_threads()
    sample = (f"per step: the {nparts} particles of the {layers}-cell slab z < {layers}/{ncell} "
              f"of the {w.name} workload, binned and interacted by the FP64 oracle")
    line = {
        "impl": "reference",
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(w, args),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config(w, args):
    return {"workload": f"{w.name}: {w.note}, uniform in [0,1)^3 (seeded), non-periodic, "
                        f"r_c={w.rc:.9g}, Gaussian K with h=r_c/2, outputs S, V and neighbour count",
            "n_particles": w.n, "cells": [w.cells_per_axis()] * 3, "r_c": w.rc, "h": w.h,
            "layout": w.layout, "algo": args.algo, "precision": args.precision,
            "parallelism": f"replicas x{args.gpus}",
            "l2": f"flushed before every timed step ({args.flush_mb} MB write)"}


# ---------------------------------------------------------------- our arm


def run_ours(args):
    import torch

    from paper_2406_16091_gb300 import binding as B
    from paper_2406_16091_gb300 import build as pibuild

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    pibuild.build()
    B.load()

    w = W.WORKLOADS[args.workload]
    # replicas: each rank runs its own independent system of the same shape
    x, y, z = W.uniform(w.n, w.seed + 1000 * rank) if w.layout == "uniform" and rank else w.positions()
    n = w.n
    s = torch.cuda.current_stream()
    ctx = B.pi_create(w.lo, w.hi, w.rc, n)
    B.pi_set_option(ctx, B.PI_OPT_ALGO, B.PI_ALGO_TILED if args.algo == "tiled" else B.PI_ALGO_PPNL)
    B.pi_set_option(ctx, B.PI_OPT_PRECISION,
                    B.PI_PREC_FP32 if args.precision == "fp32" else B.PI_PREC_KAHAN)
    tx, ty, tz = (torch.from_numpy(a).to(dev) for a in (x, y, z))
    S, Vx, Vy, Vz = (torch.empty(n, device=dev) for _ in range(4))
    nb = torch.empty(n, dtype=torch.int32, device=dev)
    flush = torch.empty(args.flush_mb * (1 << 20) // 4, device=dev)

    def step():
        B.pi_bin(ctx, tx, ty, tz, n, s)
        B.pi_interact(ctx, w.h, S, Vx, Vy, Vz, nb, B.PI_ORDER_SORTED, s)

    for _ in range(max(3, args.warmup)):
        step()
    st, mpc = B.pi_sync_status(ctx, s)
    pairs = int(nb.to(torch.int64).sum().item())

    props = torch.cuda.get_device_properties(dev)
    bus = None
    try:
        bus = f"{props.pci_domain_id:08x}:{props.pci_bus_id:02x}:{props.pci_device_id:02x}.0"
    except AttributeError:
        pass
    sampler = ClockSampler(bus)

    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    launches0 = B.pi_launch_count(ctx)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.start()
    wall0 = time.perf_counter()
    for i in range(K):
        flush.fill_(float(i))  # L2 flush between timed steps (not timed)
        e0, e1, e2 = ev[i]
        e0.record(s)
        B.pi_bin(ctx, tx, ty, tz, n, s)
        e1.record(s)
        B.pi_interact(ctx, w.h, S, Vx, Vy, Vz, nb, B.PI_ORDER_SORTED, s)
        e2.record(s)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clocks = sampler.stop()
    launches = B.pi_launch_count(ctx) - launches0
    st, mpc2 = B.pi_sync_status(ctx, s)
    t_step = [e[0].elapsed_time(e[2]) * 1e-3 for e in ev]
    t_bin = [e[0].elapsed_time(e[1]) * 1e-3 for e in ev]
    t_int = [e[1].elapsed_time(e[2]) * 1e-3 for e in ev]
    dev_time = sum(t_step)
    if ws > 1:
        import torch.distributed as dist

        tt = torch.tensor([dev_time], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        dev_time_max = float(tt.item())
        pt = torch.tensor([pairs], dtype=torch.float64, device=dev)
        dist.all_reduce(pt, op=dist.ReduceOp.SUM)
        pairs_all = float(pt.item())
    else:
        dev_time_max = dev_time
        pairs_all = float(pairs)
    value = pairs_all * K / dev_time_max

    # ---- end to end through the host-buffer entry point (pinned memory)
    e2e = None
    if args.e2e_steps > 0:
        hx, hy, hz = (torch.from_numpy(a).pin_memory() for a in (x, y, z))
        hout = [torch.empty(n).pin_memory() for _ in range(4)]
        hnb = torch.empty(n, dtype=torch.int32).pin_memory()
        for _ in range(3):
            B.pi_run_host(ctx, hx, hy, hz, n, w.h, *hout, hnb, B.PI_ORDER_SORTED, s)
        te = []
        for _ in range(args.e2e_steps):
            t0 = time.perf_counter()
            B.pi_run_host(ctx, hx, hy, hz, n, w.h, *hout, hnb, B.PI_ORDER_SORTED, s)
            te.append(time.perf_counter() - t0)
        e2e_pairs = int(hnb.numpy().astype(np.int64).sum())
        t_e2e = sum(te)
        if ws > 1:
            import torch.distributed as dist

            tt = torch.tensor([t_e2e, float(e2e_pairs)], dtype=torch.float64, device=dev)
            mx = tt.clone()
            dist.all_reduce(mx, op=dist.ReduceOp.MAX)
            dist.all_reduce(tt, op=dist.ReduceOp.SUM)
            t_e2e, e2e_pairs_all = float(mx[0]), float(tt[1])
        else:
            e2e_pairs_all = float(e2e_pairs)
        e2e = {"value": e2e_pairs_all * args.e2e_steps / t_e2e, "unit": UNIT,
               "h2d_bytes_per_step": 3 * 4 * n, "d2h_bytes_per_step": 5 * 4 * n,
               "ms_per_step": 1e3 * t_e2e / args.e2e_steps, "steps": args.e2e_steps,
               "api": "pi_run_host (pinned host buffers)"}
    B.pi_destroy(ctx)

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return

    peaks, peak_kind = measured_peaks()
    sms = props.multi_processor_count
    sm_max = float(peaks.get("sm_max_mhz") or (clocks or {}).get("sm_max_mhz") or 2070.0)
    alu_peak = sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12  # TFLOP/s
    mean_int = statistics.fmean(t_int)
    achieved = FLOP_PER_PAIR * pairs / mean_int / 1e12
    src = os.path.join(ROOT, "paper_2406_16091_gb300", "csrc")
    kname = "k_interact_tiled" if args.algo == "tiled" else "k_interact_ppnl"
    traffic = recorded_traffic(kname, source_hash([os.path.join(src, "pi_interact.cu"),
                                                   os.path.join(src, "pi_internal.cuh")]))
    roofline = {
        "kernel": kname, "bound": "alu", "achieved": achieved, "peak": alu_peak,
        "unit": "TFLOP/s", "frac": achieved / alu_peak,
        "traffic": traffic["dram_bytes_per_launch"] if traffic else None,
        "algorithmic_flop_per_launch": FLOP_PER_PAIR * pairs,
        "algorithmic_bytes_per_launch": 36 * n + 4 * (w.cells_per_axis() ** 3 + 1),
        "mean_launch_us": 1e6 * mean_int,
        "peak_basis": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 FLOP x {sm_max:.0f} MHz",
    }
    if clocks:
        roofline["frac_at_median_clock"] = achieved / (alu_peak * clocks["sm_mhz"] / sm_max)
    C = w.cells_per_axis() ** 3
    bin_bytes = 72 * n + 12 * C
    mean_bin = statistics.fmean(t_bin)
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    binning = {"bound": "hbm", "achieved": bin_bytes / mean_bin / 1e9, "peak": hbm_peak,
               "unit": "GB/s", "frac": bin_bytes / mean_bin / 1e9 / hbm_peak,
               "algorithmic_bytes": bin_bytes, "mean_us": 1e6 * mean_bin,
               "kernels": ["k_zero", "k_hist", "k_scan", "k_scatter", "k_stabilise"]}

    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        import oracle

        oracle.build()
        t0 = time.perf_counter()
        b = oracle.bin_particles(x, y, z, w.lo, w.hi, w.rc)
        r = oracle.interact(b, w.rc, w.h)
        t_cpu = time.perf_counter() - t0
        cpu = {"value": int(r.nbr.sum()) / t_cpu, "unit": UNIT, "cores": oracle.num_threads(),
               "kind": "oracle",
               "sample": f"one full step (bin + interact) of the {w.name} workload, "
                         f"{n} particles, FP64 oracle, {t_cpu:.2f} s"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K,
        "warmup": args.warmup, "ms_per_step": 1e3 * dev_time / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(w, args),
        "full_step_particles_per_s": ws * n * K / dev_time_max,
        "pairs_per_step": pairs, "max_per_cell": mpc2,
        "interact_pairs_per_s": pairs / mean_int, "bin_us": 1e6 * mean_bin,
        "interact_us": 1e6 * mean_int,
        "roofline": roofline, "roofline_binning": binning, "peak_source": peak_kind,
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
        "clocks": clocks, "timed_region_wall_s": wall,
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

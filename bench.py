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

from paper_2406_16091_gb300 import replicas  # noqa: E402
from paper_2406_16091_gb300 import workloads as W  # noqa: E402

METRIC = "within-cutoff pair interactions/s"
UNIT = "pairs/s"
# FLOP per within-cutoff ordered pair in the per-target formulation:
# 3 (displacement) + 5 (r^2) + 1 (scale) + 1 (exp2) + 1 (S) + 6 (V)
FLOP_PER_PAIR = 17
FP32_LANES_PER_SM = 128
# The binning paths (PI_OPT_BINNING values of include/pi.h), their kernels
# and the sources whose DRAM bytes profiles/traffic.json records.
BINNING_PATHS = {
    "per_particle": {"option": 0, "traffic_key": "binning", "files": ["pi_bin.cu", "pi_internal.cuh"],
                     "kernels": ["k_zero", "k_hist", "k_scan", "k_scatter", "k_stabilise"]},
    "bucketed": {"option": 1, "traffic_key": "binning_bucketed",
                 "files": ["pi_bin.cu", "pi_bucket.cu", "pi_internal.cuh"],
                 "kernels": ["k_zero", "k_bucket_count", "k_scan", "k_bucket_scatter", "k_bucket_cells",
                             "k_bucket_big"]},
    "radix": {"option": 2, "traffic_key": "binning_radix", "files": ["pi_bin.cu", "pi_radix.cu", "pi_internal.cuh"],
              "kernels": ["k_zero", "k_radix_keys", "k_scan", "k_radix_scatter", "k_radix_count",
                          "k_radix_gather", "k_radix_rank"]},
}


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
    p.add_argument("--e2e-in-flight", type=int, default=6,
                   help="contexts (and streams) the end-to-end steps rotate over")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--flush-mb", type=int, default=512)
    p.add_argument("--tile", default="auto", choices=["auto", "0", "1", "2", "3", "4", "5", "6"],
                   help="tile shape of the tiled interaction (auto: pi_autotune during warm-up)")
    p.add_argument("--study", choices=["none", "precision", "batched", "serving", "sweep", "sizes"],
                   default="none", help="run one of the extra studies instead of the main line")
    p.add_argument("--jobs", type=int, default=10000, help="serving study: number of jobs")
    p.add_argument("--max-slots", type=int, default=8, help="serving study: slots per capacity bucket")
    p.add_argument("--binning", choices=list(BINNING_PATHS), default="per_particle",
                   help="binning path (PI_OPT_BINNING)")
    p.add_argument("--no-extras", action="store_true",
                   help="leave out the batched, serving and per-configuration records of the line")
    p.add_argument("--serving-jobs", type=int, default=1000,
                   help="jobs of the line's serving record (Poisson arrivals at 80 %% of capacity)")
    return p.parse_args()


def binning_bytes(n, C):
    """Algorithmic bytes of binning a1-a4: per particle 12 read + 4 cell +
    4 rank written (a1/a2), 8 read (cell, rank) + 12 read (x, y, z) + 4 perm
    + 12 sorted positions written (a4); per cell 4 (count clear) + 4 read +
    4 written (a3)."""
    return 48 * n + 12 * C


def binning_bytes_with_p(n, C):
    """binning_bytes plus what this library's binning also writes for the
    interaction: the 16-byte x-ordered P record per particle, and its 8-byte
    per-cell sub-bin word (reported beside the algorithmic figure)."""
    return 48 * n + 16 * n + 12 * C + 8 * C


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            return d, "measured"
        except Exception:
            pass
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def evaluations_per_pair(B, ctx, step, pairs, s):
    """Target-source evaluations per within-cutoff pair of one step, counted by
    the direct kernels (PI_OPT_COUNT_EVALS) in an untimed step; None for the
    shapes that do not count."""
    B.pi_set_option(ctx, B.PI_OPT_COUNT_EVALS, 1)
    try:
        step()
        e = B.pi_eval_count(ctx, s)
    finally:
        B.pi_set_option(ctx, B.PI_OPT_COUNT_EVALS, 0)
    return e / pairs if e and pairs else None


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
    return {"workload": f"{w.name}: {w.note}, {w.layout} in [0,1)^3 (seeded), non-periodic, "
                        f"r_c={w.rc:.9g}, Gaussian K with h=r_c/2, outputs S, V and neighbour count",
            "n_particles": w.n, "cells": [w.cells_per_axis()] * 3, "r_c": w.rc, "h": w.h,
            "layout": w.layout, "algo": args.algo, "precision": args.precision,
            "binning": getattr(args, "binning", "per_particle"),
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
    x, y, z = replicas.replica_positions(w, rank)
    n = w.n
    s = torch.cuda.current_stream()
    ctx = B.pi_create(w.lo, w.hi, w.rc, n)
    B.pi_set_option(ctx, B.PI_OPT_ALGO, B.PI_ALGO_TILED if args.algo == "tiled" else B.PI_ALGO_PPNL)
    B.pi_set_option(ctx, B.PI_OPT_PRECISION,
                    B.PI_PREC_FP32 if args.precision == "fp32" else B.PI_PREC_KAHAN)
    B.pi_set_option(ctx, B.PI_OPT_BINNING, BINNING_PATHS[args.binning]["option"])
    tx, ty, tz = (torch.from_numpy(a).to(dev) for a in (x, y, z))
    S, Vx, Vy, Vz = (torch.empty(n, device=dev) for _ in range(4))
    nb = torch.empty(n, dtype=torch.int32, device=dev)
    flush = torch.empty(args.flush_mb * (1 << 20) // 4, device=dev)

    def step():
        B.pi_bin(ctx, tx, ty, tz, n, s)
        B.pi_interact(ctx, w.h, S, Vx, Vy, Vz, nb, B.PI_ORDER_SORTED, s)

    tile_ms, tile = None, None
    if args.algo == "tiled" and args.tile == "auto":
        # the autotuner may also pick Alg. 1 (PPNL); the line reports the choice
        step()
        tile, tile_ms = B.pi_autotune(ctx, [w.h], S, Vx, Vy, Vz, nb, B.PI_ORDER_SORTED, 5, s)
        if tile == B.PI_AUTOTUNE_PPNL:
            args.algo = "ppnl"
    elif args.algo == "tiled":
        tile = int(args.tile)
        B.pi_set_option(ctx, B.PI_OPT_TILE, tile)
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
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(K)]
    launches0 = B.pi_launch_count(ctx)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.start()
    wall0 = time.perf_counter()
    for i in range(K):
        flush.fill_(float(i))  # L2 flush between timed steps (not timed)
        e0, e2 = ev[i]
        # no event between binning and interaction: it would keep the
        # interaction from launching while the binning's last kernel drains
        e0.record(s)
        step()
        e2.record(s)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clocks = sampler.stop()
    launches = B.pi_launch_count(ctx) - launches0
    st, mpc2 = B.pi_sync_status(ctx, s)
    t_step = [e[0].elapsed_time(e[1]) * 1e-3 for e in ev]
    dev_time = sum(t_step)

    # the split between binning and interaction, from separate steps with an
    # event between the two (not part of the timed region above)
    KB = min(K, 1000)
    evb = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(KB)]
    for i in range(KB):
        flush.fill_(float(i))
        e0, e1, e2 = evb[i]
        e0.record(s)
        B.pi_bin(ctx, tx, ty, tz, n, s)
        e1.record(s)
        B.pi_interact(ctx, w.h, S, Vx, Vy, Vz, nb, B.PI_ORDER_SORTED, s)
        e2.record(s)
    torch.cuda.synchronize()
    t_bin = [e[0].elapsed_time(e[1]) * 1e-3 for e in evb]
    t_int = [e[1].elapsed_time(e[2]) * 1e-3 for e in evb]
    dev_time_max, pairs_all = replicas.aggregate(dev_time, pairs, dev)
    value = replicas.job_rate(pairs_all, K, dev_time_max)

    # the paper's protocol: the mean of 200 back-to-back asynchronous
    # interaction calls (no L2 flush between them)
    eb0, eb1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    eb0.record(s)
    for _ in range(200):
        B.pi_interact(ctx, w.h, S, Vx, Vy, Vz, nb, B.PI_ORDER_SORTED, s)
    eb1.record(s)
    eb1.synchronize()
    back_to_back = 1e3 * eb0.elapsed_time(eb1) / 200
    # evaluations per useful pair, counted in one more (untimed) step
    evals = evaluations_per_pair(B, ctx, step, pairs, s)

    # ---- end to end through the host-buffer entry points (pinned memory)
    e2e = None
    try:
        if args.e2e_steps > 0:
            hx, hy, hz = (torch.from_numpy(a).pin_memory() for a in (x, y, z))
            hout = [torch.empty(n).pin_memory() for _ in range(4)]
            hnb = torch.empty(n, dtype=torch.int32).pin_memory()
            # (1) blocking: one pi_run_host per step
            for _ in range(3):
                B.pi_run_host(ctx, hx, hy, hz, n, w.h, *hout, hnb, B.PI_ORDER_SORTED, s)
            te = []
            for _ in range(args.e2e_steps):
                t0 = time.perf_counter()
                B.pi_run_host(ctx, hx, hy, hz, n, w.h, *hout, hnb, B.PI_ORDER_SORTED, s)
                te.append(time.perf_counter() - t0)
            e2e_pairs = int(hnb.numpy().astype(np.int64).sum())
            t_e2e, e2e_pairs_all = replicas.aggregate(sum(te), e2e_pairs, dev)
            blocking = {"value": replicas.job_rate(e2e_pairs_all, args.e2e_steps, t_e2e), "unit": UNIT,
                        "ms_per_step": 1e3 * t_e2e / args.e2e_steps, "steps": args.e2e_steps,
                        "api": "pi_run_host (pinned host buffers), one blocking call per step"}
            # (2) pipelined: steps rotate over PIPE contexts on their own streams
            # through pi_submit_host_strided (positions in one pinned block, one
            # copy in; outputs into one pinned block, one copy out), so one
            # step's copies and latency-bound binning overlap the others'
            # kernels.  Every step copies its positions in and its outputs out.
            PIPE = max(1, args.e2e_in_flight)
            d = (n + 3) // 4 * 4
            hin = torch.empty(3 * d).pin_memory()
            for k, a_ in enumerate((x, y, z)):
                hin[k * d:k * d + n] = torch.from_numpy(a_)
            ib = hin.data_ptr()
            ctxs = [ctx] + [B.pi_create(w.lo, w.hi, w.rc, n) for _ in range(PIPE - 1)]
            for c in ctxs[1:]:
                B.pi_set_option(c, B.PI_OPT_ALGO, B.PI_ALGO_TILED if args.algo == "tiled" else B.PI_ALGO_PPNL)
                B.pi_set_option(c, B.PI_OPT_PRECISION,
                                B.PI_PREC_FP32 if args.precision == "fp32" else B.PI_PREC_KAHAN)
                if args.algo == "tiled":
                    B.pi_set_option(c, B.PI_OPT_TILE, tile)
            streams = [torch.cuda.Stream(dev) for _ in range(PIPE)]
            houts = [torch.empty(5 * d).pin_memory() for _ in range(PIPE)]

            def submit(k):
                c = k % PIPE
                ob = houts[c].data_ptr()
                B.pi_submit_host_strided(ctxs[c], w.lo, w.hi, w.rc, ib, ib + 4 * d, ib + 8 * d, d, n, w.h,
                                         *(ob + 4 * d * j for j in range(5)), d, B.PI_ORDER_SORTED,
                                         streams[c])

            for k in range(2 * PIPE):
                submit(k)
            torch.cuda.synchronize()
            K2 = max(PIPE, args.e2e_steps)
            t0 = time.perf_counter()
            for k in range(K2):
                submit(k)
            torch.cuda.synchronize()
            t_pipe = time.perf_counter() - t0
            for c in range(PIPE):
                B.pi_sync_status(ctxs[c], streams[c])
            nbr_last = houts[(K2 - 1) % PIPE][4 * d:4 * d + n].view(torch.int32)
            pipe_pairs = int(nbr_last.numpy().astype(np.int64).sum())
            assert pipe_pairs == e2e_pairs, "the contexts disagree on the pair count"
            t_pipe, pipe_pairs_all = replicas.aggregate(t_pipe, pipe_pairs, dev)
            e2e = {"value": replicas.job_rate(pipe_pairs_all, K2, t_pipe), "unit": UNIT,
                   "h2d_bytes_per_step": 3 * 4 * n, "d2h_bytes_per_step": 5 * 4 * n,
                   "ms_per_step": 1e3 * t_pipe / K2, "steps": K2, "steps_in_flight": PIPE,
                   "api": f"pi_submit_host_strided (pinned host blocks), steps rotating over {PIPE} "
                          "contexts on their own streams; every step copies its positions in and its "
                          "outputs out",
                   "blocking": blocking}
            for c in ctxs[1:]:
                B.pi_destroy(c)
    except Exception as exc:  # the line is still printed
        print(f"bench: end-to-end measurement failed: {exc!r}", file=sys.stderr)
        e2e = {"error": repr(exc)}

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
    if args.algo != "tiled":
        kname = "k_interact_ppnl"
    else:
        kname = {3: "k_interact_ws", 4: "k_interact_ws", 5: "k_interact_direct",
                 6: "k_interact_direct4"}.get(tile, "k_interact_tiled")
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
        "evaluations_per_useful_pair": evals,
    }
    if clocks:
        roofline["frac_at_median_clock"] = achieved / (alu_peak * clocks["sm_mhz"] / sm_max)
    C = w.cells_per_axis() ** 3
    bin_bytes = binning_bytes(n, C)
    bin_path = BINNING_PATHS[args.binning]
    bin_kernels = bin_path["kernels"]
    mean_bin = statistics.fmean(t_bin)
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    # the DRAM bytes of the binning path that ran (its kernels' sources)
    bin_traffic = recorded_traffic(bin_path["traffic_key"],
                                   source_hash([os.path.join(src, f) for f in bin_path["files"]]))
    bin_dram = bin_traffic["dram_bytes_per_launch"] if bin_traffic else None
    binning = {"bound": "hbm", "achieved": bin_bytes / mean_bin / 1e9, "peak": hbm_peak,
               "unit": "GB/s", "frac": bin_bytes / mean_bin / 1e9 / hbm_peak,
               "algorithmic_bytes": bin_bytes,
               "algorithmic_bytes_formula": "48 N + 12 C (a1-a4 per particle and per cell)",
               "bytes_with_P_record": binning_bytes_with_p(n, C), "mean_us": 1e6 * mean_bin,
               "traffic": bin_dram,
               "traffic_over_algorithmic": bin_dram / bin_bytes if bin_dram else None,
               "kernels": bin_kernels}

    # the other parts of the metric and the other configurations, measured
    # after the timed region: batched systems, served jobs, per configuration
    extras = {}
    if not args.no_extras and ws == 1:
        for key, fn in (("per_config", lambda: per_config_records(torch, B, args.flush_mb, alu_peak, hbm_peak)),
                        ("batched", lambda: batched_record(torch, B, args.flush_mb, 10, 5)),
                        ("serving", lambda: serving_record(torch, B, args.serving_jobs, args.max_slots,
                                                           loads=(0.8,)))):
            t0 = time.perf_counter()
            try:
                extras[key] = fn()
            except Exception as exc:  # the line is still printed
                print(f"bench: {key} record failed: {exc!r}", file=sys.stderr)
                extras[key] = {"error": repr(exc)}
            extras[key]["wall_s"] = time.perf_counter() - t0

    cpu = None
    try:
        if not args.no_cpu_baseline and ws == 1:
            import oracle

            oracle.build()
            # whole oracle steps on the same particles, repeated for about 10 s
            reps, t_bin_cpu, t_int_cpu, cpu_pairs = 0, 0.0, 0.0, 0
            while reps == 0 or t_bin_cpu + t_int_cpu < 10.0:
                t0 = time.perf_counter()
                b = oracle.bin_particles(x, y, z, w.lo, w.hi, w.rc)
                t1 = time.perf_counter()
                r = oracle.interact(b, w.rc, w.h)
                t_bin_cpu += t1 - t0
                t_int_cpu += time.perf_counter() - t1
                cpu_pairs += int(r.nbr.sum())
                reps += 1
            t_cpu = t_bin_cpu + t_int_cpu
            cores = oracle.num_threads()
            # and one step on a single core
            oracle.set_num_threads(1)
            try:
                t0 = time.perf_counter()
                b = oracle.bin_particles(x, y, z, w.lo, w.hi, w.rc)
                r1 = oracle.interact(b, w.rc, w.h)
                t_one = time.perf_counter() - t0
            finally:
                oracle.set_num_threads(cores)
            cpu = {"value": cpu_pairs / t_cpu, "unit": UNIT, "cores": cores,
                   "kind": "oracle",
                   "sample": f"{reps} full steps (bin + interact) of the {w.name} workload, "
                             f"{n} particles each, FP64 oracle, {t_cpu:.1f} s in all",
                   "bin_s_per_step": t_bin_cpu / reps, "interact_s_per_step": t_int_cpu / reps,
                   "single_core": {"value": int(r1.nbr.sum()) / t_one, "unit": UNIT, "s_per_step": t_one}}
    except Exception as exc:  # the line is still printed
        print(f"bench: oracle baseline failed: {exc!r}", file=sys.stderr)
        cpu = {"error": repr(exc)}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K,
        "warmup": args.warmup, "ms_per_step": 1e3 * dev_time / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(w, args),
        "full_step_particles_per_s": ws * n * K / dev_time_max,
        "pairs_per_step": pairs, "max_per_cell": mpc2,
        "interact_pairs_per_s": pairs / mean_int, "bin_us": 1e6 * mean_bin,
        "interact_us": 1e6 * mean_int, "split_steps": KB, "bin_us_median": 1e6 * statistics.median(t_bin),
        "interact_us_median": 1e6 * statistics.median(t_int),
        "interact_us_back_to_back": back_to_back,
        "tile": tile, "tile_ms": tile_ms,
        "roofline": roofline, "roofline_binning": binning, "peak_source": peak_kind,
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
        "clocks": clocks, "timed_region_wall_s": wall,
        **extras,
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()



# ---------------------------------------------------------------- studies
#
# Extra measurements, one JSON line each ("study": name).  They are not the
# benchmark line the contract above defines; they cover the other workloads:
# the precision study (clustered workload, FP32 vs Kahan vs the FP64 oracle),
# the batched workload (many uneven systems in one launch vs one launch set
# per system), the serving workload (Poisson arrivals) and a sweep of
# occupancy, interaction kernel and algorithm.


def _torch_setup():
    import torch

    from paper_2406_16091_gb300 import binding as B
    from paper_2406_16091_gb300 import build as pibuild

    torch.cuda.set_device(0)
    pibuild.build()
    B.load()
    return torch, B


def _time_events(torch, fn, reps, flush=None):
    """Median and mean milliseconds of fn() over reps runs (CUDA events on the
    current stream), with an optional L2 flush before each run."""
    s = torch.cuda.current_stream()
    ts = []
    for i in range(reps):
        if flush is not None:
            flush.fill_(float(i))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        fn()
        e1.record(s)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts), statistics.fmean(ts)


def study_precision(args):
    """Clustered workload: the sums of plain FP32 and of Kahan-compensated
    FP32 accumulation against the FP64 oracle, error stated per output, plus
    the FP64 GPU totals of V (which vanish up to rounding)."""
    import oracle

    torch, B = _torch_setup()
    w = W.WORKLOADS["clustered"]
    x, y, z = w.positions()
    dev = torch.device("cuda", 0)
    t0 = time.perf_counter()
    b = oracle.bin_particles(x, y, z, w.lo, w.hi, w.rc)
    r = oracle.interact(b, w.rc, w.h)
    t_oracle = time.perf_counter() - t0
    ctx = B.pi_create(w.lo, w.hi, w.rc, w.n)
    s = torch.cuda.current_stream()
    tx, ty, tz = (torch.from_numpy(a).to(dev) for a in (x, y, z))
    out = [torch.empty(w.n, device=dev) for _ in range(4)]
    nb = torch.empty(w.n, dtype=torch.int32, device=dev)
    tot = torch.zeros(1, dtype=torch.float64, device=dev)
    res = {"study": "precision", "workload": "clustered: " + w.note, "n": w.n,
           "pairs": int(r.nbr.sum()), "oracle_seconds": t_oracle, "oracle_threads": oracle.num_threads()}
    B.pi_bin(ctx, tx, ty, tz, w.n, s)
    for name, prec in (("fp32", B.PI_PREC_FP32), ("kahan", B.PI_PREC_KAHAN)):
        B.pi_set_option(ctx, B.PI_OPT_PRECISION, prec)
        B.pi_interact(ctx, w.h, *out, nb, B.PI_ORDER_SORTED, s)
        B.pi_sync_status(ctx, s)
        ms, _ = _time_events(torch, lambda: B.pi_interact(ctx, w.h, *out, nb, B.PI_ORDER_SORTED, s), 10)
        entry = {"interact_ms": ms,
                 "nbr_exact": bool(np.array_equal(nb.cpu().numpy().view(np.uint32), r.nbr))}
        for k, (o, ref, ab) in enumerate(zip(out, (r.S, r.Vx, r.Vy, r.Vz),
                                             (r.absS, r.absVx, r.absVy, r.absVz))):
            g = o.cpu().numpy().astype(np.float64)
            nz = ab > 0
            rel = np.abs(g[nz] - ref[nz]) / ab[nz]
            key = ("S", "Vx", "Vy", "Vz")[k]
            entry[key] = {"max_rel": float(rel.max()), "mean_rel": float(rel.mean()),
                          "p99_rel": float(np.percentile(rel, 99)),
                          "max_abs": float(np.abs(g - ref).max())}
            if k > 0:
                B.pi_total_f64(ctx, o, tot, s)
                entry[key]["gpu_fp64_total"] = float(tot.cpu()[0])
                entry[key]["total_over_sum_abs"] = abs(float(tot.cpu()[0])) / float(ab.sum())
        res[name] = entry
    B.pi_destroy(ctx)
    print(json.dumps(res), flush=True)


def batched_record(torch, B, flush_mb, reps_batch=20, reps_plain=10):
    """The batched workload: 256 uneven systems in one context (one launch per
    kernel, graph-captured, tile shape autotuned) against one context and one
    launch set per system, at the same accuracy (bitwise-equal outputs)."""
    dev = torch.device("cuda", 0)
    systems = W.batched_systems()
    ns = [sy.n for sy in systems]
    N = sum(ns)
    pos = [sy.positions() for sy in systems]
    cat = lambda k: torch.from_numpy(np.concatenate([p[k] for p in pos])).to(dev)
    tx, ty, tz = cat(0), cat(1), cat(2)
    hs = [sy.h for sy in systems]
    s = torch.cuda.current_stream()
    flush = torch.empty(flush_mb * (1 << 20) // 4, device=dev)
    # --- batched
    ctx = B.pi_batch_create([(sy.lo, sy.hi) for sy in systems], [sy.rc for sy in systems], ns)
    out = [torch.empty(N, device=dev) for _ in range(4)]
    nb = torch.empty(N, dtype=torch.int32, device=dev)
    B.pi_batch_bin(ctx, tx, ty, tz, ns, s)
    tile, tile_ms = B.pi_autotune(ctx, hs, *out, nb, B.PI_ORDER_SORTED, 5, s)

    def step_batch():
        B.pi_batch_bin(ctx, tx, ty, tz, ns, s)
        B.pi_batch_interact(ctx, hs, *out, nb, B.PI_ORDER_SORTED, s)

    for _ in range(3):
        step_batch()
    pairs = int(nb.to(torch.int64).sum().item())
    ms_batch, _ = _time_events(torch, step_batch, reps_batch, flush)
    g = torch.cuda.CUDAGraph()
    cs = torch.cuda.Stream()
    cs.wait_stream(s)
    with torch.cuda.stream(cs):
        step_batch_cs = lambda: (B.pi_batch_bin(ctx, tx, ty, tz, ns, cs),
                                 B.pi_batch_interact(ctx, hs, *out, nb, B.PI_ORDER_SORTED, cs))
        step_batch_cs()
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=cs):
            step_batch_cs()
    s.wait_stream(cs)
    ms_graph, _ = _time_events(torch, g.replay, reps_batch, flush)
    B.pi_sync_status(ctx, s)
    batch_out = [o.clone() for o in out] + [nb.clone()]
    # --- one context per system, launched one after the other
    ctxs = [B.pi_create(sy.lo, sy.hi, sy.rc, sy.n) for sy in systems]
    offs = np.concatenate([[0], np.cumsum(ns)])
    views = lambda t, k: t[int(offs[k]):int(offs[k + 1])]

    def step_plain(stream=s):
        for k, c in enumerate(ctxs):
            B.pi_bin(c, views(tx, k), views(ty, k), views(tz, k), ns[k], stream)
            B.pi_interact(c, hs[k], *[views(o, k) for o in out], views(nb, k), B.PI_ORDER_SORTED, stream)

    for _ in range(3):
        step_plain()
    ms_plain, _ = _time_events(torch, step_plain, reps_plain, flush)
    g2 = torch.cuda.CUDAGraph()
    with torch.cuda.stream(cs):
        step_plain(cs)
        torch.cuda.synchronize()
        with torch.cuda.graph(g2, stream=cs):
            step_plain(cs)
    s.wait_stream(cs)
    ms_plain_graph, _ = _time_events(torch, g2.replay, reps_plain, flush)
    torch.cuda.synchronize()
    same = all(torch.equal(a.view(torch.int32), b.view(torch.int32))
               for a, b in zip(batch_out, [o for o in out] + [nb]))
    for c in ctxs:
        B.pi_destroy(c)
    B.pi_destroy(ctx)
    res = {"study": "batched", "systems": len(systems), "particles": N, "pairs": pairs,
           "tile_chosen": tile, "tile_ms": tile_ms,
           "batched_ms": ms_batch, "batched_graph_ms": ms_graph,
           "plain_ms": ms_plain, "plain_graph_ms": ms_plain_graph,
           "batched_graph_pairs_per_s": pairs / (ms_graph * 1e-3),
           "plain_pairs_per_s": pairs / (ms_plain * 1e-3),
           "speedup_vs_plain": ms_plain / ms_graph,
           "speedup_vs_plain_graph": ms_plain_graph / ms_graph,
           "outputs_bitwise_equal": bool(same),
           "l2": "flushed before every timed step"}
    return res


def study_batched(args):
    torch, B = _torch_setup()
    print(json.dumps(batched_record(torch, B, args.flush_mb)), flush=True)


def serving_record(torch, B, n_jobs, max_slots, loads=(0.5, 0.8, 0.95)):
    """The serving workload: jobs of N log-uniform in [1k, 1M], occupancy in
    {2, 4, 8, 16}, half uniform and half clustered.  First the capacity (all
    jobs queued at once), then the same jobs one after another as blocking
    pi_run_host calls (the plain per-system loop), then Poisson arrivals at
    the given fractions of the capacity."""
    from paper_2406_16091_gb300.serving import Server, make_job

    specs = W.serving_jobs(n_jobs)
    t0 = time.perf_counter()
    pool = {k: [torch.from_numpy(a).pin_memory() for a in v] for k, v in W.serving_pool().items()}
    jobs = []
    for k, sp in enumerate(specs):
        x, y, z = (a[: sp.n] for a in pool[sp.layout])
        # results of every 500th job are kept; the others land in slot buffers
        jobs.append(make_job(k, x, y, z, sp.lo, sp.hi, sp.rc, sp.h, outputs=k % 500 == 0))
    t_gen = time.perf_counter() - t0
    srv = Server(buckets=((65536, 4), (262144, 4), (1048576, 2)), max_slots_per_bucket=max_slots)
    res = {"study": "serving", "jobs": len(jobs), "particles": sum(j.n for j in jobs),
           "generation_s": t_gen}
    try:
        # warm-up: every slot once
        warm = jobs[: min(20, len(jobs))]
        for j in warm:
            j.arrival = 0.0
        srv.run(warm)
        for j in jobs:
            j.arrival = 0.0
        cap = srv.run(jobs)
        res["capacity"] = cap
        # the plain queue: the same jobs one after another, each a blocking
        # pi_run_host on one context sized for the largest job
        ctx = B.pi_create((0, 0, 0), (1, 1, 1), W.rc_for_cells(int(round(
            max(j.cells for j in jobs) ** (1 / 3))) + 1), max(j.n for j in jobs))
        try:
            hout = [torch.empty(max(j.n for j in jobs)).pin_memory() for _ in range(4)]
            hnb = torch.empty(max(j.n for j in jobs), dtype=torch.int32).pin_memory()
            s0 = torch.cuda.current_stream()
            B.pi_run_host(ctx, hout[0], hout[0], hout[0], 0, 0.5, *hout, hnb, B.PI_ORDER_ORIGINAL, s0)
            t1 = time.perf_counter()
            for j in jobs:
                B.pi_reconfigure(ctx, j.lo, j.hi, j.rc, s0)
                B.pi_run_host(ctx, j.x, j.y, j.z, j.n, j.h, *hout, hnb, B.PI_ORDER_ORIGINAL, s0)
            t_plain = time.perf_counter() - t1
        finally:
            B.pi_destroy(ctx)
        res["plain_sequential"] = {"jobs_per_s": len(jobs) / t_plain,
                                   "particles_per_s": sum(j.n for j in jobs) / t_plain,
                                   "makespan_s": t_plain}
        res["speedup_vs_plain"] = cap["jobs_per_s"] / res["plain_sequential"]["jobs_per_s"]
        rng = np.random.default_rng(1005)
        for frac in loads:
            rate = frac * cap["jobs_per_s"]
            t = np.cumsum(rng.exponential(1.0 / rate, len(jobs)))
            for j, a in zip(jobs, t):
                j.arrival = float(a)
            res[f"load_{int(frac * 100)}"] = srv.run(jobs)
    finally:
        srv.close()
    return res


def study_serving(args):
    torch, B = _torch_setup()
    print(json.dumps(serving_record(torch, B, args.jobs, args.max_slots)), flush=True)


def per_config_records(torch, B, flush_mb, alu_peak, hbm_peak=6800.0,
                       names=("scale_ppc1", "scale_ppc2", "scale_ppc4", "scale_ppc16", "scale_ppc32",
                              "clustered"),
                       reps=20):
    """The other single-GPU configurations: per workload one full step and the
    interaction alone (medians of CUDA events, L2 flushed before each), with
    the shape pi_autotune picks, the within-cutoff pairs per second, the
    interaction's fraction of the FP32 peak on useful FLOP and, for the
    low-occupancy rows where its arithmetic intensity is below the FP32/HBM
    balance, its fraction of the HBM bandwidth on algorithmic bytes (36 per
    particle + 4 per cell)."""
    dev = torch.device("cuda", 0)
    flush = torch.empty(flush_mb * (1 << 20) // 4, device=dev)
    s = torch.cuda.current_stream()
    rows = {}
    for name in names:
        w = W.WORKLOADS[name]
        x, y, z = w.positions()
        ctx = B.pi_create(w.lo, w.hi, w.rc, w.n)
        try:
            t = [torch.from_numpy(a).to(dev) for a in (x, y, z)]
            out = [torch.empty(w.n, device=dev) for _ in range(4)]
            nb = torch.empty(w.n, dtype=torch.int32, device=dev)
            B.pi_bin(ctx, *t, w.n, s)
            chosen, _ = B.pi_autotune(ctx, [w.h], *out, nb, B.PI_ORDER_SORTED, 3, s)
            B.pi_sync_status(ctx, s)
            pairs = int(nb.to(torch.int64).sum().item())
            inter = lambda: B.pi_interact(ctx, w.h, *out, nb, B.PI_ORDER_SORTED, s)
            step = lambda: (B.pi_bin(ctx, *t, w.n, s), inter())
            step()
            int_ms, _ = _time_events(torch, inter, reps, flush)
            step_ms, _ = _time_events(torch, step, reps, flush)
            _, mpc = B.pi_sync_status(ctx, s)
            evals = evaluations_per_pair(B, ctx, step, pairs, s)
            rows[name] = {"n": w.n, "cells_per_axis": w.cells_per_axis(), "layout": w.layout,
                          "max_per_cell": mpc, "pairs": pairs,
                          "shape": "ppnl" if chosen == B.PI_AUTOTUNE_PPNL else f"tile{chosen}",
                          "step_ms": step_ms, "interact_ms": int_ms,
                          "pairs_per_s": pairs / (step_ms * 1e-3),
                          "interact_pairs_per_s": pairs / (int_ms * 1e-3),
                          "full_step_particles_per_s": w.n / (step_ms * 1e-3),
                          "interact_frac_of_fp32_peak": FLOP_PER_PAIR * pairs / (int_ms * 1e-3) / 1e12 / alu_peak,
                          "interact_frac_of_hbm": (36 * w.n + 4 * (w.cells_per_axis() ** 3 + 1))
                          / (int_ms * 1e-3) / 1e9 / hbm_peak,
                          "evaluations_per_useful_pair": evals}
            del t, out, nb
        finally:
            B.pi_destroy(ctx)
    return {"rows": rows, "timing": f"medians of {reps} CUDA-event timings, L2 flushed before each",
            "frac_basis": "17 FLOP per within-cutoff ordered pair over the derived FP32 peak"}


def study_sweep(args):
    """Interaction throughput over occupancy (1-32 particles per cell), over
    the interaction kernels of Sec. 7.1-7.2, and the tiled kernel's speedup
    over Par-Part-NoLoop (Alg. 1) -- the paper's comparison."""
    torch, B = _torch_setup()
    dev = torch.device("cuda", 0)
    flush = torch.empty(args.flush_mb * (1 << 20) // 4, device=dev)
    s = torch.cuda.current_stream()
    rows = []
    names = ["scale_ppc1", "scale_ppc2", "scale_ppc4", "scale", "scale_ppc16", "scale_ppc32"]
    kernels = [("gaussian", B.PI_KERNEL_GAUSSIAN), ("lj", B.PI_KERNEL_LJ),
               ("lowflop", B.PI_KERNEL_LOWFLOP), ("highflop", B.PI_KERNEL_HIGHFLOP)]
    for name in names:
        w = W.WORKLOADS[name]
        x, y, z = w.positions()
        ctx = B.pi_create(w.lo, w.hi, w.rc, w.n)
        t = [torch.from_numpy(a).to(dev) for a in (x, y, z)]
        out = [torch.empty(w.n, device=dev) for _ in range(4)]
        nb = torch.empty(w.n, dtype=torch.int32, device=dev)
        B.pi_bin(ctx, *t, w.n, s)
        B.pi_sync_status(ctx, s)
        for kname, kern in kernels if name == "scale" else kernels[:1]:
            B.pi_set_option(ctx, B.PI_OPT_KERNEL, kern)
            entry = {"workload": name, "kernel": kname}
            run = lambda: B.pi_interact(ctx, w.h, *out, nb, B.PI_ORDER_SORTED, s)
            for algo_name, algo in (("tiled", B.PI_ALGO_TILED), ("ppnl", B.PI_ALGO_PPNL)):
                B.pi_set_option(ctx, B.PI_OPT_ALGO, algo)
                B.pi_set_option(ctx, B.PI_OPT_TILE, 5)
                run()
                ms, _ = _time_events(torch, run, 10, flush)
                entry[f"{algo_name}_ms"] = ms
            # what the autotuner picks for this occupancy and kernel
            chosen, cand_ms = B.pi_autotune(ctx, [w.h], *out, nb, B.PI_ORDER_SORTED, 3, s)
            entry["autotuned"] = "ppnl" if chosen == B.PI_AUTOTUNE_PPNL else f"tile{chosen}"
            entry["autotuned_ms"], _ = _time_events(torch, run, 10, flush)
            entry["candidate_ms"] = cand_ms
            pairs = int(nb.to(torch.int64).sum().item())
            entry["pairs"] = pairs
            entry["tiled_pairs_per_s"] = pairs / (entry["tiled_ms"] * 1e-3)
            entry["autotuned_pairs_per_s"] = pairs / (entry["autotuned_ms"] * 1e-3)
            entry["speedup_vs_ppnl"] = entry["ppnl_ms"] / entry["tiled_ms"]
            rows.append(entry)
        B.pi_set_option(ctx, B.PI_OPT_KERNEL, B.PI_KERNEL_GAUSSIAN)
        B.pi_set_option(ctx, B.PI_OPT_ALGO, B.PI_ALGO_TILED)
        B.pi_sync_status(ctx, s)
        B.pi_destroy(ctx)
    print(json.dumps({"study": "sweep", "rows": rows}), flush=True)


def study_sizes(args):
    """One full step (bin + interact) at 8 particles per cell from 32 K to
    2^28 particles (the largest about 20 GB on the device): throughput in N,
    medians of CUDA events with the L2 flushed before every step."""
    torch, B = _torch_setup()
    dev = torch.device("cuda", 0)
    flush = torch.empty(args.flush_mb * (1 << 20) // 4, device=dev)
    s = torch.cuda.current_stream()
    rows = []
    for n in (1 << 15, 1 << 18, 1 << 21, 1 << 24, 1 << 26, 1 << 28):
        w = W.scaled(W.SCALE, n)
        x, y, z = w.positions()
        ctx = B.pi_create(w.lo, w.hi, w.rc, n)
        try:
            tx, ty, tz = (torch.from_numpy(a).to(dev) for a in (x, y, z))
            out = [torch.empty(n, device=dev) for _ in range(4)]
            nb = torch.empty(n, dtype=torch.int32, device=dev)
            B.pi_bin(ctx, tx, ty, tz, n, s)
            B.pi_interact(ctx, w.h, *out, nb, B.PI_ORDER_SORTED, s)
            B.pi_sync_status(ctx, s)
            pairs = int(nb.to(torch.int64).sum().item())
            reps = 20 if n <= (1 << 24) else 5
            bin_ms, _ = _time_events(torch, lambda: B.pi_bin(ctx, tx, ty, tz, n, s), reps, flush)
            step_ms, _ = _time_events(torch, lambda: (B.pi_bin(ctx, tx, ty, tz, n, s),
                                                      B.pi_interact(ctx, w.h, *out, nb, B.PI_ORDER_SORTED, s)),
                                      reps, flush)
            B.pi_sync_status(ctx, s)
            rows.append({"n": n, "cells_per_axis": w.cells_per_axis(), "pairs": pairs,
                         "step_ms": step_ms, "bin_ms": bin_ms,
                         "pairs_per_s": pairs / (step_ms * 1e-3),
                         "particles_per_s": n / (step_ms * 1e-3)})
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
            del tx, ty, tz, out, nb
        finally:
            B.pi_destroy(ctx)
        torch.cuda.empty_cache()
    print(json.dumps({"study": "sizes", "rows": rows, "l2": "flushed before every timed step"}), flush=True)


STUDIES = {"precision": study_precision, "batched": study_batched, "serving": study_serving,
           "sweep": study_sweep, "sizes": study_sizes}

def main():
    args = parse()
    if args.study != "none":
        STUDIES[args.study](args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

"""Host side of the multi-GPU form: independent replicas.

The method has no data exchange between GPUs that this library performs:
every rank (one process per GPU) bins and interacts its own system, and the
job's throughput is the work of all ranks divided by the slowest rank's time
(weak scaling).  This module holds that logic so that it can be tested with
CPU process groups (``gloo``); the benchmark runs it over NCCL.
"""
from __future__ import annotations

from . import workloads as W


def replica_positions(w: W.Workload, rank: int):
    """Positions of ``rank``'s system: the workload itself on rank 0, an
    independent draw of the same shape (same N, box, cutoff and layout, seed
    shifted by 1000 per rank) on the others."""
    if rank == 0:
        return w.positions()
    seed = w.seed + 1000 * rank
    if w.layout == "clustered":
        return W.clustered(w.n, seed)
    return W.uniform(w.n, seed, w.lo, w.hi)


def aggregate(local_time_s: float, local_units: float, device=None):
    """(max over ranks of the time, sum over ranks of the units) through
    ``torch.distributed`` (all-reduce MAX and SUM); the local values when no
    process group is initialised.  ``device``: where the reduction tensors
    live (a CUDA device for NCCL, the CPU for gloo)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(local_time_s), float(local_units)
    t = torch.tensor([float(local_time_s)], dtype=torch.float64, device=device)
    u = torch.tensor([float(local_units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def job_rate(units_all: float, steps: int, time_max_s: float) -> float:
    """Whole-job throughput: units of all ranks per step times the steps,
    over the slowest rank's time."""
    if time_max_s <= 0:
        raise ValueError("time must be positive")
    return units_all * steps / time_max_s

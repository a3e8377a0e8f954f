"""Continuous-batching server for cutoff-interaction jobs on one GPU.

Jobs (host positions, box, cutoff, kernel width) arrive over time.  The
request loop itself is native (``pi_server_run`` in the C library): it
keeps device-resident contexts ("slots"), each with its own CUDA stream,
completion event and pinned scratch block, and enqueues a job on a free slot
with one ``pi_submit_host_strided`` call, which re-targets the slot's grid
to the job's box and cutoff (no allocation), copies the positions in, bins,
interacts and copies the results out.  A job's grid thus lives on the
device only while it runs, and the next job reuses it.

Admission is continuous: whenever a slot is free, the oldest waiting job
that fits it is started at once, so the work of several jobs overlaps on the
GPU while the host keeps admitting and completing.  Slots come in capacity
buckets; a job waits in the queue of the smallest bucket that fits it and
may also take a free slot of a larger bucket.  When every slot that fits a
job is busy and the device still has memory within the server's HBM budget,
a new slot is created (memory-based admission); otherwise the job waits.
Completion is polled through CUDA events.

Every job runs exactly the kernels a lone ``pi_bin`` + ``pi_interact``
would run, on its own slot, so its results do not depend on the mix.  This
module builds the job records and reports the statistics.
"""
from __future__ import annotations

import ctypes
import time
from dataclasses import dataclass, field

import numpy as np

from . import binding as B


@dataclass
class Job:
    """One request.  Inputs are pinned host tensors (x, y, z; with
    in_stride > 0 they are views of one block, y = x + in_stride and z = x +
    2 in_stride); the outputs (S, Vx, Vy, Vz, nbr) are pinned host tensors
    filled by the server (views of one block when out_stride > 0), or None:
    the results then land in the slot's scratch block, which the slot's next
    job overwrites (for callers that consume a result as soon as the job
    completes)."""
    jid: int
    n: int
    lo: tuple
    hi: tuple
    rc: float
    h: float
    x: object
    y: object
    z: object
    arrival: float = 0.0
    S: object = None
    Vx: object = None
    Vy: object = None
    Vz: object = None
    nbr: object = None
    t_start: float = 0.0
    t_done: float = 0.0
    cells: int = 0
    in_stride: int = 0
    out_stride: int = 0
    blocks: list = field(default_factory=list)  # keeps the pinned blocks alive


def job_cells(lo, hi, rc) -> int:
    """Cells of a job's grid (the grid rule of pi_create, in FP64)."""
    c = 1
    for d in range(3):
        c *= max(1, int(np.floor((float(hi[d]) - float(lo[d])) / float(rc))))
    return c


def _stride(n: int) -> int:
    return max(4, (int(n) + 3) // 4 * 4)


def make_job(jid, x, y, z, lo, hi, rc, h, arrival=0.0, outputs=True):
    """A job from host positions: numpy arrays are copied into one pinned
    block (one host-to-device copy per job); pinned torch tensors are used
    as they are.  ``outputs``: allocate the job's own pinned result block."""
    import torch

    n = len(x)
    d = _stride(n)
    job = Job(jid=jid, n=n, lo=tuple(lo), hi=tuple(hi), rc=float(rc), h=float(h), x=None, y=None, z=None,
              arrival=float(arrival), cells=job_cells(lo, hi, rc))
    if isinstance(x, torch.Tensor):
        job.x, job.y, job.z = x, y, z
    else:
        blk = torch.empty(3 * d).pin_memory()
        for k, a in enumerate((x, y, z)):
            blk[k * d: k * d + n] = torch.from_numpy(np.ascontiguousarray(a, np.float32))
        job.x, job.y, job.z = blk[0:n], blk[d:d + n], blk[2 * d:2 * d + n]
        job.in_stride = d
        job.blocks.append(blk)
    if outputs:
        out = torch.empty(5 * d).pin_memory()
        job.S, job.Vx, job.Vy, job.Vz = (out[k * d: k * d + n] for k in range(4))
        job.nbr = out[4 * d: 4 * d + n].view(torch.int32)
        job.out_stride = d
        job.blocks.append(out)
    return job


def slot_bytes(n_cap: int, c_cap: int | None = None) -> int:
    """Device memory one slot of particle capacity n_cap is charged against
    the server's HBM budget (cell capacity = particle capacity)."""
    return B.pi_server_slot_bytes(n_cap)


class Server:
    """Continuous-batching server over the native request loop.
    ``buckets``: (particle capacity, initial slots) per bucket, cell capacity
    = particle capacity; ``hbm_budget``: bytes the slots may occupy (default:
    half of the free device memory)."""

    def __init__(self, buckets=((65536, 2), (262144, 2), (1048576, 1)), hbm_budget=None,
                 max_slots_per_bucket=8, device=0):
        import torch

        self.device = torch.device("cuda", device)
        caps = [int(b[0]) for b in buckets]
        init = [int(b[1]) for b in buckets]
        with torch.cuda.device(self.device):
            self.srv = B.pi_server_create(caps, init, max_slots_per_bucket,
                                          0 if hbm_budget is None else int(hbm_budget))
        self.caps = sorted(caps)

    def bucket_of(self, job: Job) -> int | None:
        """Smallest bucket whose slots fit the job, None if none does."""
        for cap in self.caps:
            if cap >= job.n and cap >= job.cells:
                return cap
        return None

    def fits(self, job: Job) -> bool:
        return self.bucket_of(job) is not None

    def run(self, jobs):
        """Serves ``jobs`` (each with an ``arrival`` offset in seconds from
        the start).  Returns statistics; every job gets its outputs, start
        and completion times (seconds from the start)."""
        import torch

        for j in jobs:
            if self.bucket_of(j) is None:
                raise ValueError(f"job {j.jid} fits no slot bucket")
        arr = (B.PiJob * len(jobs))()
        for r, j in zip(arr, jobs):
            r.n = int(j.n)
            if j.n > 0:  # (an empty job copies nothing: no addresses)
                r.x, r.y, r.z = B._ptr(j.x), B._ptr(j.y), B._ptr(j.z)
                r.in_stride = int(j.in_stride)
            r.box = B.PiBox((ctypes.c_float * 3)(*j.lo), (ctypes.c_float * 3)(*j.hi))
            r.r_c, r.h = float(j.rc), float(j.h)
            if j.S is not None and j.n > 0:
                r.S, r.Vx, r.Vy, r.Vz = B._ptr(j.S), B._ptr(j.Vx), B._ptr(j.Vy), B._ptr(j.Vz)
                r.nbr = B._ptr(j.nbr)
                r.out_stride = int(j.out_stride)
            r.arrival = float(j.arrival)
        with torch.cuda.device(self.device):
            makespan = B.pi_server_run(self.srv, arr)
        for r, j in zip(arr, jobs):
            j.t_start, j.t_done = r.t_start, r.t_done
        caps, slots, used = B.pi_server_info(self.srv)
        lat = np.array([j.t_done - j.arrival for j in jobs])
        return {"jobs": len(jobs), "makespan_s": makespan, "jobs_per_s": len(jobs) / makespan,
                "particles_per_s": sum(j.n for j in jobs) / makespan,
                "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                "mean_ms": 1e3 * float(lat.mean()),
                "slots": dict(zip(caps, slots)),
                "hbm_used_bytes": used}

    def close(self):
        if self.srv is not None:
            B.pi_server_destroy(self.srv)
            self.srv = None

"""Continuous-batching server for cutoff-interaction jobs on one GPU.

Jobs (host positions, box, cutoff, kernel width) arrive over time.  The
server keeps device-resident contexts ("slots"), each with its own CUDA
stream and device staging buffers; a job is enqueued on a free slot with one
call, ``pi_submit_host``, which re-targets the slot's grid to the job's box
and cutoff (no allocation), copies the positions in, bins, interacts and
copies the results out.  A job's grid thus lives on the device only while it
runs, and the next job reuses it.

Admission is continuous: whenever a slot is free, the oldest waiting job
that fits it is started at once, so the work of several jobs overlaps on the
GPU while the host keeps admitting and completing.  Slots come in capacity
buckets; a job waits in the queue of the smallest bucket that fits it and
may also take a free slot of a larger bucket.  When every slot that fits a
job is busy and the device still has memory within the server's HBM budget,
a new slot is created (memory-based admission); otherwise the job waits.
Completion is polled through CUDA events.

Every job runs exactly the kernels a lone ``pi_bin`` + ``pi_interact``
would run, on its own slot, so its results do not depend on the mix.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass

import numpy as np

from . import binding as B
from .workloads import rc_for_cells


@dataclass
class Job:
    """One request.  Inputs are pinned host tensors (x, y, z); the outputs
    (S, Vx, Vy, Vz, nbr) are pinned host tensors filled by the server, or
    None: the results then land in the slot's own host buffers, which the
    next job on that slot overwrites (for callers that consume a result as
    soon as the job completes)."""
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


def job_cells(lo, hi, rc) -> int:
    """Cells of a job's grid (the grid rule of pi_create, in FP64)."""
    c = 1
    for d in range(3):
        c *= max(1, int(np.floor((float(hi[d]) - float(lo[d])) / float(rc))))
    return c


def make_job(jid, x, y, z, lo, hi, rc, h, arrival=0.0, outputs=True):
    """A job from host positions (numpy arrays, copied to pinned memory, or
    pinned torch tensors, used as they are); ``outputs``: allocate the job's
    own pinned result buffers."""
    import torch

    n = len(x)

    def pin(a):
        if isinstance(a, torch.Tensor):
            return a
        return torch.from_numpy(np.ascontiguousarray(a, np.float32)).pin_memory()

    job = Job(jid=jid, n=n, lo=tuple(lo), hi=tuple(hi), rc=float(rc), h=float(h), x=pin(x),
              y=pin(y), z=pin(z), arrival=float(arrival), cells=job_cells(lo, hi, rc))
    if outputs:
        out = [torch.empty(max(n, 1)).pin_memory() for _ in range(4)]
        job.S, job.Vx, job.Vy, job.Vz = out
        job.nbr = torch.empty(max(n, 1), dtype=torch.int32).pin_memory()
    return job


def slot_bytes(n_cap: int, c_cap: int) -> int:
    """Device memory of one slot: the context arena (72 bytes per particle,
    about 28 per cell) plus its host-transfer staging buffers (32 bytes per
    particle); an upper estimate."""
    return int(n_cap) * (80 + 32) + int(c_cap) * 32 + (1 << 20)


class Slot:
    def __init__(self, n_cap: int, c_cap: int, device, bucket: int):
        import torch

        self.n_cap, self.c_cap, self.bucket = int(n_cap), int(c_cap), int(bucket)
        # a unit box with k^3 >= c_cap cells sizes the grid capacity
        k = int(np.ceil(c_cap ** (1.0 / 3.0) - 1e-9))
        self.ctx = B.pi_create((0, 0, 0), (1, 1, 1), rc_for_cells(k), self.n_cap)
        self.stream = torch.cuda.Stream(device=device)
        # host results of jobs without their own buffers
        self.hout = [torch.empty(self.n_cap).pin_memory() for _ in range(4)]
        self.hnb = torch.empty(self.n_cap, dtype=torch.int32).pin_memory()
        self.event = torch.cuda.Event()
        self.job: Job | None = None
        # allocate the staging buffers now, outside the request loop
        z = torch.zeros(1).pin_memory()
        B.pi_submit_host(self.ctx, (0, 0, 0), (1, 1, 1), rc_for_cells(k), z, z, z, 0, 0.5,
                         *self.hout, self.hnb, B.PI_ORDER_ORIGINAL, self.stream)
        self.stream.synchronize()

    def start(self, job: Job, now: float):
        job.t_start = now
        own = job.S is not None
        outs = (job.S, job.Vx, job.Vy, job.Vz) if own else self.hout
        B.pi_submit_host(self.ctx, job.lo, job.hi, job.rc, job.x, job.y, job.z, job.n, job.h, *outs,
                         job.nbr if own else self.hnb, B.PI_ORDER_ORIGINAL, self.stream)
        self.event.record(self.stream)
        self.job = job

    def destroy(self):
        B.pi_destroy(self.ctx)


class Server:
    """Continuous-batching server.  ``buckets``: (particle capacity, initial
    slots) per bucket, cell capacity = particle capacity; ``hbm_budget``:
    bytes the slots may occupy (default: half of the free device memory)."""

    def __init__(self, buckets=((65536, 2), (262144, 2), (1048576, 1)), hbm_budget=None,
                 max_slots_per_bucket=8, device=0):
        import torch

        self.device = torch.device("cuda", device)
        free, _ = torch.cuda.mem_get_info(self.device)
        self.budget = int(hbm_budget if hbm_budget is not None else free // 2)
        self.used = 0
        self.caps = sorted(int(b[0]) for b in buckets)
        self.max_per_bucket = int(max_slots_per_bucket)
        self.slots = {c: [] for c in self.caps}
        self.free = {c: [] for c in self.caps}
        for cap, k in buckets:
            for _ in range(k):
                s = self._grow(int(cap))
                if s is not None:
                    self.free[s.bucket].append(s)

    def _grow(self, cap: int) -> Slot | None:
        """New slot of a bucket if it fits the bucket's limit, the HBM budget
        and the device's free memory (checked in that order)."""
        import torch

        if len(self.slots[cap]) >= self.max_per_bucket:
            return None
        need = slot_bytes(cap, cap)
        if self.used + need > self.budget:
            return None
        free, _ = torch.cuda.mem_get_info(self.device)
        if need > free:
            return None
        s = Slot(cap, cap, self.device, cap)
        self.slots[cap].append(s)
        self.used += need
        return s

    def bucket_of(self, job: Job) -> int | None:
        """Smallest bucket whose slots fit the job, None if none does."""
        for cap in self.caps:
            if cap >= job.n and cap >= job.cells:
                return cap
        return None

    def fits(self, job: Job) -> bool:
        return self.bucket_of(job) is not None

    def _admit(self, queues, busy, now):
        """Starts waiting jobs while slots are free or can be created: for
        each bucket from the largest down, its free slots take the oldest
        job among the queues of that bucket and the smaller ones."""
        for bi in range(len(self.caps) - 1, -1, -1):
            cap = self.caps[bi]
            while True:
                # oldest head among the queues this bucket can serve
                best = None
                for bj in range(bi + 1):
                    q = queues[self.caps[bj]]
                    if q and (best is None or q[0].arrival < queues[best][0].arrival):
                        best = self.caps[bj]
                if best is None:
                    break
                if not self.free[cap]:
                    s = self._grow(cap)
                    if s is None:
                        break
                    self.free[cap].append(s)
                slot = self.free[cap].pop()
                slot.start(queues[best].popleft(), now)
                busy.append(slot)

    def run(self, jobs, clock=time.perf_counter):
        """Serves ``jobs`` (each with an ``arrival`` offset in seconds from
        the start).  Returns statistics; every job gets its outputs, start
        and completion times (seconds from the start)."""
        for j in jobs:
            if self.bucket_of(j) is None:
                raise ValueError(f"job {j.jid} fits no slot bucket")
        pending = deque(sorted(jobs, key=lambda j: j.arrival))
        queues = {c: deque() for c in self.caps}
        busy: list[Slot] = []
        done = 0
        total = len(pending)
        t0 = clock()
        while done < total:
            now = clock() - t0
            arrived = False
            while pending and pending[0].arrival <= now:
                j = pending.popleft()
                queues[self.bucket_of(j)].append(j)
                arrived = True
            # completions
            freed = False
            still = []
            for s in busy:
                if s.event.query():
                    s.job.t_done = clock() - t0
                    s.job = None
                    self.free[s.bucket].append(s)
                    done += 1
                    freed = True
                else:
                    still.append(s)
            busy = still
            if arrived or freed:
                self._admit(queues, busy, clock() - t0)
            if not busy and pending and not any(queues.values()):
                wait = pending[0].arrival - (clock() - t0)
                if wait > 0:
                    time.sleep(min(wait, 0.001))
        makespan = clock() - t0
        for s in (s for lst in self.slots.values() for s in lst):
            st, _ = B.pi_sync_status(s.ctx, s.stream, raise_on_error=False)
            if st != B.PI_OK:
                raise B.PiError(st, "serving")
        lat = np.array([j.t_done - j.arrival for j in jobs])
        return {"jobs": total, "makespan_s": makespan, "jobs_per_s": total / makespan,
                "particles_per_s": sum(j.n for j in jobs) / makespan,
                "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                "mean_ms": 1e3 * float(lat.mean()),
                "slots": {c: len(v) for c, v in self.slots.items()},
                "hbm_used_bytes": self.used}

    def close(self):
        for lst in self.slots.values():
            for s in lst:
                s.destroy()
        self.slots = {c: [] for c in self.caps}
        self.free = {c: [] for c in self.caps}

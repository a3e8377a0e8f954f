"""Continuous-batching server for cutoff-interaction jobs on one GPU.

Jobs (host positions, box, cutoff, kernel width) arrive over time.  The
server keeps device-resident contexts ("slots"), each with its own CUDA
stream and its own device input/output buffers; a slot is re-targeted to a
job's box and cutoff with ``pi_reconfigure`` (no allocation), so a job's
grid lives on the device only while it runs and the next job reuses it.

Admission is continuous: whenever a slot is free, the oldest waiting job
that fits it is started at once -- host-to-device copy, binning,
interaction and device-to-host copy are enqueued on the slot's stream, so
the work of several jobs overlaps on the GPU while the host keeps admitting
and completing.  Slots come in capacity buckets; when every slot that fits
a job is busy and the device still has free memory within the server's HBM
budget, a new slot is created (memory-based admission); otherwise the job
waits.  Completion is polled through CUDA events.

Every job runs exactly the kernels a lone ``pi_bin`` + ``pi_interact``
would run, on its own buffers, so its results do not depend on the mix.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import binding as B
from .workloads import rc_for_cells


@dataclass
class Job:
    """One request.  Inputs are pinned host tensors (x, y, z); the outputs
    (S, Vx, Vy, Vz, nbr) are pinned host tensors filled by the server."""
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
    status: int = B.PI_OK


def make_job(jid, x, y, z, lo, hi, rc, h, arrival=0.0):
    import torch

    n = len(x)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).pin_memory()
    out = [torch.empty(max(n, 1)).pin_memory() for _ in range(4)]
    nb = torch.empty(max(n, 1), dtype=torch.int32).pin_memory()
    return Job(jid=jid, n=n, lo=tuple(lo), hi=tuple(hi), rc=float(rc), h=float(h), x=pin(x),
               y=pin(y), z=pin(z), arrival=float(arrival), S=out[0], Vx=out[1], Vy=out[2],
               Vz=out[3], nbr=nb)


def slot_bytes(n_cap: int, c_cap: int) -> int:
    """Device memory of one slot: the context arena plus the slot's own
    input/output buffers (an upper estimate)."""
    return int(n_cap) * (76 + 32) + int(c_cap) * 24 + (1 << 20)


class Slot:
    def __init__(self, n_cap: int, c_cap: int, device):
        import torch

        self.n_cap, self.c_cap = int(n_cap), int(c_cap)
        # a unit box with k^3 >= c_cap cells sizes the grid capacity
        k = int(np.ceil(c_cap ** (1.0 / 3.0) - 1e-9))
        self.ctx = B.pi_create((0, 0, 0), (1, 1, 1), rc_for_cells(k), self.n_cap)
        self.stream = torch.cuda.Stream(device=device)
        self.x, self.y, self.z = (torch.empty(self.n_cap, device=device) for _ in range(3))
        self.out = [torch.empty(self.n_cap, device=device) for _ in range(4)]
        self.nb = torch.empty(self.n_cap, dtype=torch.int32, device=device)
        self.event = torch.cuda.Event()
        self.job: Job | None = None

    def start(self, job: Job, now: float):
        import torch

        n = job.n
        s = self.stream
        job.t_start = now
        with torch.cuda.stream(s):
            if n:
                self.x[:n].copy_(job.x[:n], non_blocking=True)
                self.y[:n].copy_(job.y[:n], non_blocking=True)
                self.z[:n].copy_(job.z[:n], non_blocking=True)
            B.pi_reconfigure(self.ctx, job.lo, job.hi, job.rc, s)
            B.pi_bin(self.ctx, self.x, self.y, self.z, n, s)
            if n:
                B.pi_interact(self.ctx, job.h, *self.out, self.nb, B.PI_ORDER_ORIGINAL, s)
                for dst, src in zip((job.S, job.Vx, job.Vy, job.Vz), self.out):
                    dst[:n].copy_(src[:n], non_blocking=True)
                job.nbr[:n].copy_(self.nb[:n], non_blocking=True)
            self.event.record(s)
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
        for cap, k in buckets:
            for _ in range(k):
                self._grow(int(cap))

    def _grow(self, cap: int) -> Slot | None:
        """New slot of a bucket if it fits the HBM budget and the device."""
        import torch

        need = slot_bytes(cap, cap)
        free, _ = torch.cuda.mem_get_info(self.device)
        if (self.used + need > self.budget or need > free
                or len(self.slots[cap]) >= self.max_per_bucket):
            return None
        s = Slot(cap, cap, self.device)
        self.slots[cap].append(s)
        self.used += need
        return s

    def _free_slot(self, job: Job, allow_grow=True) -> Slot | None:
        cells = 1
        for d in range(3):
            cells *= max(1, int(np.floor((job.hi[d] - job.lo[d]) / job.rc)))
        for cap in self.caps:
            if cap < job.n or cap < cells:
                continue
            for s in self.slots[cap]:
                if s.job is None:
                    return s
        if allow_grow:
            for cap in self.caps:
                if cap >= job.n and cap >= cells:
                    s = self._grow(cap)
                    if s is not None:
                        return s
        return None

    def fits(self, job: Job) -> bool:
        return any(c >= job.n for c in self.caps)

    def run(self, jobs, clock=time.perf_counter):
        """Serves ``jobs`` (each with an ``arrival`` offset in seconds from
        the start).  Returns statistics; every job gets its outputs, start
        and completion times (seconds from the start)."""
        pending = deque(sorted(jobs, key=lambda j: j.arrival))
        waiting: deque[Job] = deque()
        busy: list[Slot] = []
        done = 0
        total = len(pending)
        t0 = clock()
        while done < total:
            now = clock() - t0
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            # completions
            still = []
            for s in busy:
                if s.event.query():
                    s.job.t_done = clock() - t0
                    s.job = None
                    done += 1
                else:
                    still.append(s)
            busy = still
            # admissions: oldest first, any job that a free slot fits
            if waiting:
                keep = deque()
                while waiting:
                    job = waiting.popleft()
                    slot = self._free_slot(job)
                    if slot is None:
                        keep.append(job)
                        continue
                    slot.start(job, clock() - t0)
                    busy.append(slot)
                waiting = keep
            if not busy and not waiting and pending:
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

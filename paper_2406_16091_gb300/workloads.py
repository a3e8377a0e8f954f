"""Seeded synthetic particle workloads.

This module only draws positions and picks the box, cutoff and kernel width
of each named workload.  It holds none of the method's arithmetic (no cell
index, no scan, no interaction), so both the CUDA path and the CPU oracle may
take their inputs from it.

The paper measures on uniform random particles in a non-periodic box with 1,
10 or 100 particles per cell on average (Sec. 7.1); the workloads below keep
that structure at GB300 sizes:

* ``small``      N = 32,768 uniform in [0,1)^3, r_c = 1/16 (16^3 cells, 8 per cell)
* ``scale``      N = 2,097,152 uniform, r_c = 1/64 (64^3 cells, 8 per cell)
* ``scale_ppcK`` the same positions with r_c picked so that there are
                 128^3, 102^3, 81^3, 51^3 or 40^3 cells (about 1, 2, 4, 16, 32
                 particles per cell)
* ``clustered``  N = 4,194,304: 10 % uniform background, 90 % split evenly over
                 64 isotropic Gaussian clusters (sigma 0.03, uniform centres),
                 r_c = 1/128; samples outside [0,1)^3 are drawn again.
* ``batched_systems``  256 independent systems, N log-uniform in [1024,
                 262144], each uniform in its own unit box with a mean
                 occupancy uniform in [2, 16] (cells per axis max(3,
                 round(cbrt(N / occupancy)))).
* ``serving_jobs``  10,000 jobs, N log-uniform in [1024, 1048576], occupancy
                 in {2, 4, 8, 16}, half uniform and half clustered; their
                 particles come from ``serving_pool``.

The kernel width is h = r_c / 2 everywhere.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def rc_for_cells(n_cells: int, length: float = 1.0) -> float:
    """Largest FP32 cutoff not above ``length / n_cells``.

    With r_c <= length / n the grid rule floor(length / r_c) gives exactly n
    cells per axis (r_c > length / (n + 1) holds for the nearest float)."""
    rc = np.float32(length / n_cells)
    while float(rc) * n_cells > length:
        rc = np.nextafter(rc, np.float32(0.0))
    return float(rc)


def uniform(n: int, seed: int, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)):
    """n FP32 positions, uniform in the half-open box [lo, hi)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for d in range(3):
        u = rng.random(n, dtype=np.float32)  # [0, 1)
        a, b = np.float32(lo[d]), np.float32(hi[d])
        v = (a + (b - a) * u).astype(np.float32)
        # rounding may land on hi: move such samples just inside the box
        v = np.where(v >= b, np.nextafter(b, a), v).astype(np.float32)
        v = np.where(v < a, a, v).astype(np.float32)
        out.append(np.ascontiguousarray(v))
    return tuple(out)


def clustered(n: int, seed: int, n_clusters: int = 64, sigma: float = 0.03,
              background: float = 0.10):
    """Gaussian clusters plus a uniform background in [0,1)^3 (FP32).

    ``background`` of the particles are uniform; the rest are split evenly
    over ``n_clusters`` isotropic normals N(centre, sigma^2 I) with uniform
    centres.  Draws outside [0,1)^3 are redrawn (truncation)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n_bg = int(round(n * background))
    n_cl = n - n_bg
    centres = rng.random((n_clusters, 3))
    sizes = np.full(n_clusters, n_cl // n_clusters, dtype=np.int64)
    sizes[: n_cl - int(sizes.sum())] += 1
    pts = [rng.random((n_bg, 3))]
    for c in range(n_clusters):
        need = int(sizes[c])
        got = []
        while need > 0:
            s = centres[c] + sigma * rng.standard_normal((need + need // 8 + 16, 3))
            s = s.astype(np.float32)
            s = s[np.all((s >= 0.0) & (s < 1.0), axis=1)][:need]
            got.append(s)
            need -= len(s)
        pts.append(np.concatenate(got))
    p = np.concatenate(pts).astype(np.float32)
    p = p[rng.permutation(len(p))]
    p = np.clip(p, 0.0, np.nextafter(np.float32(1.0), np.float32(0.0)))
    return tuple(np.ascontiguousarray(p[:, d]) for d in range(3))


@dataclass
class Workload:
    name: str
    n: int
    rc: float
    h: float
    seed: int
    layout: str = "uniform"
    lo: tuple = (0.0, 0.0, 0.0)
    hi: tuple = (1.0, 1.0, 1.0)
    note: str = ""
    extra: dict = field(default_factory=dict)

    def positions(self):
        if self.layout == "uniform":
            return uniform(self.n, self.seed, self.lo, self.hi)
        if self.layout == "clustered":
            return clustered(self.n, self.seed)
        raise ValueError(self.layout)

    def cells_per_axis(self) -> int:
        return int(np.floor((self.hi[0] - self.lo[0]) / self.rc))


def _wl(name, n, cells, seed, layout="uniform", note=""):
    rc = rc_for_cells(cells)
    return Workload(name=name, n=n, rc=rc, h=float(np.float32(rc) / np.float32(2.0)),
                    seed=seed, layout=layout, note=note)


SMALL = _wl("small", 32768, 16, 1001, note="N=32768, 16^3 cells, ~8 per cell")
SCALE = _wl("scale", 2097152, 64, 1002, note="N=2097152, 64^3 cells, ~8 per cell")
SCALE_VARIANTS = {
    ppc: _wl(f"scale_ppc{ppc}", 2097152, cells, 1002,
             note=f"N=2097152, {cells}^3 cells, ~{ppc} per cell")
    for ppc, cells in ((1, 128), (2, 102), (4, 81), (16, 51), (32, 40))
}
CLUSTERED = _wl("clustered", 4194304, 128, 1003, layout="clustered",
                note="N=4194304, 128^3 cells, 64 Gaussian clusters + 10% background")

WORKLOADS = {w.name: w for w in [SMALL, SCALE, *SCALE_VARIANTS.values(), CLUSTERED]}


def scaled(w: Workload, n: int, seed: int | None = None) -> Workload:
    """Same layout and particles-per-cell as ``w`` with ``n`` particles: the
    cells per axis are scaled by (n / w.n)^(1/3) (at least 1)."""
    cells = max(1, int(round(w.cells_per_axis() * (n / w.n) ** (1.0 / 3.0))))
    return _wl(f"{w.name}@{n}", n, cells, w.seed if seed is None else seed, w.layout)


@dataclass
class System:
    """One independent system of a batch or one serving job."""
    n: int
    rc: float
    h: float
    seed: int
    layout: str = "uniform"
    lo: tuple = (0.0, 0.0, 0.0)
    hi: tuple = (1.0, 1.0, 1.0)

    def positions(self):
        if self.layout == "clustered":
            return clustered(self.n, self.seed)
        return uniform(self.n, self.seed, self.lo, self.hi)


def _system_for(n: int, ppc: float, seed: int, layout: str = "uniform") -> System:
    cells = max(3, int(round((n / ppc) ** (1.0 / 3.0))))
    rc = rc_for_cells(cells)
    return System(n=n, rc=rc, h=float(np.float32(rc) / np.float32(2.0)), seed=seed, layout=layout)


def batched_systems(count: int = 256, seed: int = 1004, n_lo: int = 1024, n_hi: int = 262144,
                    ppc_lo: float = 2.0, ppc_hi: float = 16.0):
    """The batched workload: ``count`` independent systems, N log-uniform in
    [n_lo, n_hi], each uniform in its own unit box with a mean occupancy
    drawn uniformly in [ppc_lo, ppc_hi] (cells per axis max(3,
    round(cbrt(N / ppc)))), h = r_c / 2."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ns = np.exp(rng.uniform(np.log(n_lo), np.log(n_hi), count)).astype(np.int64)
    ppc = rng.uniform(ppc_lo, ppc_hi, count)
    return [_system_for(int(ns[k]), float(ppc[k]), seed * 1000 + k) for k in range(count)]


def serving_pool(n: int = 1048576, seed: int = 1006):
    """Positions the serving jobs draw from: one uniform and one clustered
    set of ``n`` particles in [0,1)^3.  A job of N particles takes the first N
    of its layout's set -- a random sample of that layout, since both sets are
    in random order -- so that 10,000 jobs need no 10,000 separate draws."""
    return {"uniform": uniform(n, seed), "clustered": clustered(n, seed + 1)}


def serving_jobs(count: int = 10000, seed: int = 1005, n_lo: int = 1024, n_hi: int = 1048576):
    """The serving workload: ``count`` jobs with N log-uniform in [n_lo, n_hi],
    mean occupancy in {2, 4, 8, 16}, half uniform and half clustered.  Arrival
    times are drawn by the caller (Poisson at a chosen rate)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ns = np.exp(rng.uniform(np.log(n_lo), np.log(n_hi), count)).astype(np.int64)
    ppc = rng.choice([2.0, 4.0, 8.0, 16.0], count)
    layout = rng.choice(["uniform", "clustered"], count)
    return [_system_for(int(ns[k]), float(ppc[k]), seed * 100000 + k, str(layout[k]))
            for k in range(count)]

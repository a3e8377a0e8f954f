"""FP64 CPU oracle for cutoff-radius pair interactions on a cell grid.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` leg of ``bench.py`` may import this
package.  It shares no code with the CUDA library (``paper_2406_16091_gb300``)
and that library never imports it.

The arithmetic lives in ``pi_oracle.c`` (plain C, built with
``-ffp-contract=off``); this module only compiles it and marshals numpy
arrays through ctypes.  Each wrapper names the passage of arXiv 2406.16091
that it follows; ``pi_oracle.c`` lists the readings taken where the paper is
silent.
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pi_oracle.c")
_LIB = os.path.join(_HERE, "libpi_oracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile ``pi_oracle.c`` into ``libpi_oracle.so`` next to it.

    OpenMP is used when the compiler supports it (the result does not depend
    on the thread count); otherwise the library is built without it.
    """
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise RuntimeError("no C compiler found to build the oracle")
    base = [cc, "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
            "-fno-fast-math", "-Wall", _SRC, "-o", _LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True, text=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True, text=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        f32 = ctypes.c_float
        L.pio_grid_dims.argtypes = [P, P, f32, P]
        L.pio_grid_dims.restype = ctypes.c_int
        L.pio_cell_index.argtypes = [P, P, P, i64, P, P, P, P]
        L.pio_cell_index.restype = ctypes.c_int
        L.pio_exclusive_scan.argtypes = [P, i64, P]
        L.pio_exclusive_scan.restype = None
        L.pio_bin.argtypes = [P, P, P, i64, P, P, P, P, P, P, P, P, P, P]
        L.pio_bin.restype = ctypes.c_int
        L.pio_interact.argtypes = [P, P, P, i64, P, P, f32, f32, ctypes.c_int] + [P] * 10
        L.pio_interact.restype = ctypes.c_int
        L.pio_brute.argtypes = [P, P, P, i64, f32, f32, ctypes.c_int, P, P, P, P, P]
        L.pio_brute.restype = ctypes.c_int
        L.pio_num_threads.argtypes = []
        L.pio_num_threads.restype = ctypes.c_int
        L.pio_set_num_threads.argtypes = [ctypes.c_int]
        L.pio_set_num_threads.restype = None
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


def num_threads() -> int:
    return lib().pio_num_threads()


def set_num_threads(n: int) -> None:
    lib().pio_set_num_threads(int(n))


def grid_dims(lo, hi, rc: float) -> tuple[int, int, int]:
    """Cells per axis, n_d = max(1, floor((hi_d - lo_d) / r_c)) (Sec. 3: cell
    width at least r_c)."""
    lo = _f32(lo)
    hi = _f32(hi)
    dims = np.zeros(3, np.int32)
    st = lib().pio_grid_dims(_p(lo), _p(hi), ctypes.c_float(rc), _p(dims))
    if st != 0:
        raise ValueError("invalid box or cutoff")
    return tuple(int(d) for d in dims)


def cell_index(x, y, z, lo, hi, dims):
    """Cell of each particle from its position (Sec. 2).  Returns
    (cell uint32[n], ok)."""
    x, y, z = _f32(x), _f32(y), _f32(z)
    lo, hi = _f32(lo), _f32(hi)
    d = np.asarray(dims, np.int32)
    cell = np.zeros(len(x), np.uint32)
    st = lib().pio_cell_index(_p(x), _p(y), _p(z), len(x), _p(lo), _p(hi), _p(d), _p(cell))
    return cell, st == 0


def exclusive_scan(counts) -> np.ndarray:
    """Exclusive prefix sum with C+1 entries, the last one the total (Fig. 1)."""
    c = np.ascontiguousarray(counts, dtype=np.uint32)
    out = np.zeros(len(c) + 1, np.uint32)
    lib().pio_exclusive_scan(_p(c), len(c), _p(out))
    return out


@dataclass
class Binned:
    dims: tuple
    counts: np.ndarray
    offsets: np.ndarray
    perm: np.ndarray
    sx: np.ndarray
    sy: np.ndarray
    sz: np.ndarray
    max_per_cell: int
    ok: bool


def bin_particles(x, y, z, lo, hi, rc: float) -> Binned:
    """Binning of Sec. 2: cell index, counts, exclusive scan, stable scatter
    into cell-sorted SoA arrays; also M_C (Sec. 5.1)."""
    x, y, z = _f32(x), _f32(y), _f32(z)
    n = len(x)
    dims = grid_dims(lo, hi, rc)
    C = dims[0] * dims[1] * dims[2]
    lo, hi = _f32(lo), _f32(hi)
    d = np.asarray(dims, np.int32)
    counts = np.zeros(C, np.uint32)
    offsets = np.zeros(C + 1, np.uint32)
    perm = np.zeros(n, np.uint32)
    sx = np.zeros(n, np.float32)
    sy = np.zeros(n, np.float32)
    sz = np.zeros(n, np.float32)
    m = np.zeros(1, np.uint32)
    st = lib().pio_bin(_p(x), _p(y), _p(z), n, _p(lo), _p(hi), _p(d), _p(counts),
                       _p(offsets), _p(perm), _p(sx), _p(sy), _p(sz), _p(m))
    return Binned(dims, counts, offsets, perm, sx, sy, sz, int(m[0]), st == 0)


@dataclass
class Interactions:
    S: np.ndarray
    Vx: np.ndarray
    Vy: np.ndarray
    Vz: np.ndarray
    nbr: np.ndarray
    absS: np.ndarray
    absVx: np.ndarray
    absVy: np.ndarray
    absVz: np.ndarray
    candidates: int


GAUSSIAN, LJ, LOWFLOP, HIGHFLOP = 0, 1, 2, 3


def interact(b: Binned, rc: float, h: float, kernel: int = GAUSSIAN) -> Interactions:
    """Per-particle sums over the clipped 27-cell stencil (Sec. 2, Sec. 3),
    in the sorted order of ``b``, FP64 accumulation.  ``kernel``: GAUSSIAN,
    LJ (Sec. 7.1, sigma = h), LOWFLOP or HIGHFLOP (Sec. 7.2)."""
    n = len(b.sx)
    out = [np.zeros(n, np.float64) for _ in range(4)]
    nbr = np.zeros(n, np.uint32)
    ab = [np.zeros(n, np.float64) for _ in range(4)]
    cand = np.zeros(1, np.uint64)
    d = np.asarray(b.dims, np.int32)
    st = lib().pio_interact(_p(b.sx), _p(b.sy), _p(b.sz), n, _p(b.offsets), _p(d),
                            ctypes.c_float(rc), ctypes.c_float(h), int(kernel),
                            *[_p(a) for a in out], _p(nbr), *[_p(a) for a in ab], _p(cand))
    if st != 0:
        raise ValueError("oracle interact: bad arguments")
    return Interactions(*out, nbr, *ab, int(cand[0]))


def brute(x, y, z, rc: float, h: float, kernel: int = GAUSSIAN):
    """O(N^2) evaluation of the definition of Sec. 2 in input order.
    Returns (S, Vx, Vy, Vz, nbr)."""
    x, y, z = _f32(x), _f32(y), _f32(z)
    n = len(x)
    out = [np.zeros(n, np.float64) for _ in range(4)]
    nbr = np.zeros(n, np.uint32)
    st = lib().pio_brute(_p(x), _p(y), _p(z), n, ctypes.c_float(rc), ctypes.c_float(h), int(kernel),
                         *[_p(a) for a in out], _p(nbr))
    if st != 0:
        raise ValueError("oracle brute: bad arguments")
    return (*out, nbr)


def unpermute(values: np.ndarray, perm: np.ndarray) -> np.ndarray:
    """Sorted order -> input order: out[perm[k]] = values[k]."""
    out = np.empty_like(values)
    out[perm] = values
    return out

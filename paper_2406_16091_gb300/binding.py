"""Thin ctypes binding of libpi (include/pi.h), same names as the C ABI.

Argument marshalling only: tensors are passed as device pointers, streams as
their CUDA handles, and every step of the path runs in libpi's kernels.  The
library is loaded from the package directory; if it is missing this module
raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libpi.so")

# status codes (pi_status)
PI_OK = 0
PI_ERR_INVALID_ARG = 1
PI_ERR_CAPACITY = 2
PI_ERR_OUT_OF_BOX = 3
PI_ERR_NOT_BINNED = 4
PI_ERR_CUDA = 5
PI_ERR_TIMEOUT = 6
PI_ERR_NOMEM = 7
PI_ERR_CHECK = 8

PI_ORDER_SORTED = 0
PI_ORDER_ORIGINAL = 1

PI_OPT_ALGO = 1
PI_OPT_PRECISION = 2
PI_OPT_WAIT_LIMIT_NS = 3
PI_OPT_TEST_WITHHOLD_SCAN = 4
PI_OPT_KERNEL = 5
PI_OPT_TILE = 6
PI_OPT_BINNING = 7
PI_OPT_COUNT_EVALS = 8  # diagnostics: the direct kernels count their evaluations
PI_BIN_PER_PARTICLE = 0  # one global atomic and one 32-byte record per particle (default)
PI_BIN_BUCKETED = 1  # buckets of cells ranked in shared memory, when they fit
PI_BIN_RADIX = 2  # a stable radix sort of the particles by cell, when it fits
PI_NUM_TILES = 7  # tile shapes of PI_OPT_TILE (see include/pi.h)
PI_AUTOTUNE_PPNL = PI_NUM_TILES  # pi_autotune's index of PI_ALGO_PPNL
PI_AUTOTUNE_REGIMES = PI_NUM_TILES + 1  # pi_autotune's index of the per-regime plan
PI_TILE_AUTO = -1  # PI_OPT_TILE default: shape by mean occupancy
PI_KERNEL_GAUSSIAN = 0
PI_KERNEL_LJ = 1
PI_KERNEL_LOWFLOP = 2
PI_KERNEL_HIGHFLOP = 3
PI_ALGO_TILED = 0
PI_ALGO_PPNL = 1
PI_PREC_FP32 = 0
PI_PREC_KAHAN = 1


class PiBox(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_float * 3), ("hi", ctypes.c_float * 3)]


class PiJob(ctypes.Structure):
    """``pi_job`` of include/pi.h: one serving request."""
    _fields_ = [("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("z", ctypes.c_void_p),
                ("in_stride", ctypes.c_int64), ("n", ctypes.c_int64), ("box", PiBox),
                ("r_c", ctypes.c_float), ("h", ctypes.c_float),
                ("S", ctypes.c_void_p), ("Vx", ctypes.c_void_p), ("Vy", ctypes.c_void_p),
                ("Vz", ctypes.c_void_p), ("nbr", ctypes.c_void_p), ("out_stride", ctypes.c_int64),
                ("arrival", ctypes.c_double), ("t_start", ctypes.c_double), ("t_done", ctypes.c_double),
                ("slot_capacity", ctypes.c_int64)]


PI_SERVER_MAX_BUCKETS = 16


class PiError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = f"{where}: {status_str(status)} ({status})"
        extra = last_error()
        if status in (PI_ERR_CUDA, PI_ERR_CHECK) and extra:
            msg += f": {extra}"
        super().__init__(msg)


class Handle:
    """A context or server handle.  ctypes passes it as the C pointer (its
    _as_parameter_); once destroyed it refuses to be passed, so a call on a
    destroyed handle raises here instead of handing freed memory to the
    library."""

    __slots__ = ("_ptr", "_what")

    def __init__(self, ptr, what: str):
        self._ptr = ptr
        self._what = what

    @property
    def _as_parameter_(self):
        if self._ptr is None:
            raise PiError(PI_ERR_INVALID_ARG, f"{self._what} used after it was destroyed")
        return ctypes.c_void_p(self._ptr)

    def _close(self):
        self._ptr = None


_lib = None


def load():
    """Loads libpi.so from the package directory (build it with
    ``paper_2406_16091_gb300.build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libpi.so is not built ({LIB_PATH}); run __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    i32, i64, f32 = ctypes.c_int, ctypes.c_int64, ctypes.c_float
    sig = {
        "pi_create": ([ctypes.POINTER(PiBox), f32, i64, ctypes.POINTER(P)], i32),
        "pi_batch_create": ([i32, ctypes.POINTER(PiBox), P, P, ctypes.POINTER(P)], i32),
        "pi_batch_bin": ([P, P, P, P, P, P], i32),
        "pi_batch_interact": ([P, P, P, P, P, P, P, i32, P], i32),
        "pi_batch_info": ([P, P, P, P], i32),
        "pi_batch_grid": ([P, i32, P], i32),
        "pi_batch_set_tiles": ([P, P], i32),
        "pi_batch_tiles": ([P, P], i32),
        "pi_destroy": ([P], i32),
        "pi_reconfigure": ([P, ctypes.POINTER(PiBox), f32, P], i32),
        "pi_bin": ([P, P, P, P, i64, P], i32),
        "pi_interact": ([P, f32, P, P, P, P, P, i32, P], i32),
        "pi_run_host": ([P, P, P, P, i64, f32, P, P, P, P, P, i32, P], i32),
        "pi_submit_host": ([P, ctypes.POINTER(PiBox), f32, P, P, P, i64, f32, P, P, P, P, P, i32, P], i32),
        "pi_submit_host_strided": ([P, ctypes.POINTER(PiBox), f32, P, P, P, i64, i64, f32, P, P, P, P, P, i64,
                                    i32, P], i32),
        "pi_server_slot_bytes": ([i64], i64),
        "pi_server_create": ([i32, P, P, i32, i64, ctypes.POINTER(P)], i32),
        "pi_server_run": ([P, ctypes.POINTER(PiJob), i64, ctypes.POINTER(ctypes.c_double)], i32),
        "pi_server_info": ([P, P, P, P, P], i32),
        "pi_server_destroy": ([P], i32),
        "pi_grid": ([P, P], i32),
        "pi_binned": ([P] + [ctypes.POINTER(P)] * 6, i32),
        "pi_copy_binned": ([P, P, P, P, P, P, P, P], i32),
        "pi_total_f64": ([P, P, P, P], i32),
        "pi_autotune": ([P, P, P, P, P, P, P, i32, i32, P, P, P], i32),
        "pi_scan_counts_noalloc": ([P, i64, P, P, P], i32),
        "pi_sync_status": ([P, P, ctypes.POINTER(ctypes.c_uint32)], i32),
        "pi_set_option": ([P, i32, i64], i32),
        "pi_launch_count": ([P, ctypes.POINTER(ctypes.c_uint64)], i32),
        "pi_eval_count": ([P, P, ctypes.POINTER(ctypes.c_uint64)], i32),
        "pi_status_str": ([i32], ctypes.c_char_p),
        "pi_last_error": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def status_str(s: int) -> str:
    return load().pi_status_str(int(s)).decode()


def last_error() -> str:
    return load().pi_last_error().decode()


def _check(st: int, where: str) -> int:
    if st != PI_OK:
        raise PiError(st, where)
    return st


def _ptr(t):
    """Device (or host) address of a tensor / array / int, or None."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    if hasattr(t, "ctypes"):
        return t.ctypes.data
    raise TypeError(type(t))


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def pi_create(lo, hi, r_c: float, n_max: int):
    box = PiBox((ctypes.c_float * 3)(*lo), (ctypes.c_float * 3)(*hi))
    out = ctypes.c_void_p()
    _check(load().pi_create(ctypes.byref(box), float(r_c), int(n_max), ctypes.byref(out)), "pi_create")
    return Handle(out.value, "context")


def pi_batch_create(boxes, r_c, n_max):
    """boxes: list of (lo, hi); r_c, n_max: one entry per system."""
    S = len(boxes)
    arr = (PiBox * S)(*[PiBox((ctypes.c_float * 3)(*lo), (ctypes.c_float * 3)(*hi)) for lo, hi in boxes])
    rc = (ctypes.c_float * S)(*[float(v) for v in r_c])
    nm = (ctypes.c_int64 * S)(*[int(v) for v in n_max])
    out = ctypes.c_void_p()
    _check(load().pi_batch_create(S, arr, ctypes.cast(rc, ctypes.c_void_p),
                                  ctypes.cast(nm, ctypes.c_void_p), ctypes.byref(out)),
           "pi_batch_create")
    return Handle(out.value, "context")


def pi_batch_bin(ctx, x, y, z, n, stream=None) -> None:
    """n: per-system particle counts (host)."""
    arr = (ctypes.c_int64 * len(n))(*[int(v) for v in n])
    _check(load().pi_batch_bin(ctx, _ptr(x), _ptr(y), _ptr(z), ctypes.cast(arr, ctypes.c_void_p),
                               _stream(stream)), "pi_batch_bin")


def pi_batch_interact(ctx, h, S, Vx, Vy, Vz, nbr=None, out_order: int = PI_ORDER_SORTED,
                      stream=None) -> None:
    """h: per-system kernel lengths (host)."""
    arr = (ctypes.c_float * len(h))(*[float(v) for v in h])
    _check(load().pi_batch_interact(ctx, ctypes.cast(arr, ctypes.c_void_p), _ptr(S), _ptr(Vx),
                                    _ptr(Vy), _ptr(Vz), _ptr(nbr), int(out_order), _stream(stream)),
           "pi_batch_interact")


def pi_batch_info(ctx):
    """(num_systems, total_cells, total_n_max)."""
    a, b, c = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
    _check(load().pi_batch_info(ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "pi_batch_info")
    return a.value, b.value, c.value


def pi_batch_grid(ctx, system: int):
    dims = (ctypes.c_int32 * 3)()
    _check(load().pi_batch_grid(ctx, int(system), ctypes.cast(dims, ctypes.c_void_p)), "pi_batch_grid")
    return tuple(dims)


def pi_batch_set_tiles(ctx, tiles) -> None:
    """Per-system tile shapes (5 or 6 each) of a batch context; None clears."""
    if tiles is None:
        _check(load().pi_batch_set_tiles(ctx, None), "pi_batch_set_tiles")
        return
    arr = (ctypes.c_int32 * len(tiles))(*[int(t) for t in tiles])
    _check(load().pi_batch_set_tiles(ctx, ctypes.cast(arr, ctypes.c_void_p)), "pi_batch_set_tiles")


def pi_batch_tiles(ctx, num_systems: int):
    """The per-system tile shapes in use (-1 each without a plan)."""
    arr = (ctypes.c_int32 * int(num_systems))()
    _check(load().pi_batch_tiles(ctx, ctypes.cast(arr, ctypes.c_void_p)), "pi_batch_tiles")
    return list(arr)


def pi_reconfigure(ctx, lo, hi, r_c: float, stream=None) -> None:
    box = PiBox((ctypes.c_float * 3)(*lo), (ctypes.c_float * 3)(*hi))
    _check(load().pi_reconfigure(ctx, ctypes.byref(box), float(r_c), _stream(stream)), "pi_reconfigure")


def pi_destroy(ctx) -> None:
    _check(load().pi_destroy(ctx), "pi_destroy")
    if isinstance(ctx, Handle):
        ctx._close()


def pi_bin(ctx, x, y, z, n: int, stream=None) -> None:
    _check(load().pi_bin(ctx, _ptr(x), _ptr(y), _ptr(z), int(n), _stream(stream)), "pi_bin")


def pi_interact(ctx, h: float, S, Vx, Vy, Vz, nbr=None, out_order: int = PI_ORDER_SORTED,
                stream=None) -> None:
    _check(load().pi_interact(ctx, float(h), _ptr(S), _ptr(Vx), _ptr(Vy), _ptr(Vz), _ptr(nbr),
                              int(out_order), _stream(stream)), "pi_interact")


def pi_run_host(ctx, x, y, z, n: int, h: float, S, Vx, Vy, Vz, nbr=None,
                out_order: int = PI_ORDER_ORIGINAL, stream=None) -> int:
    """Host arrays in and out; returns the step's status (raises on error)."""
    return _check(load().pi_run_host(ctx, _ptr(x), _ptr(y), _ptr(z), int(n), float(h), _ptr(S),
                                     _ptr(Vx), _ptr(Vy), _ptr(Vz), _ptr(nbr), int(out_order),
                                     _stream(stream)), "pi_run_host")


def pi_submit_host(ctx, lo, hi, r_c: float, x, y, z, n: int, h: float, S, Vx, Vy, Vz, nbr=None,
                   out_order: int = PI_ORDER_ORIGINAL, stream=None) -> None:
    """One job from host arrays to host arrays, enqueued on `stream` without
    waiting (re-targets the context to the box and cutoff first if needed)."""
    box = PiBox((ctypes.c_float * 3)(*lo), (ctypes.c_float * 3)(*hi))
    _check(load().pi_submit_host(ctx, ctypes.byref(box), float(r_c), _ptr(x), _ptr(y), _ptr(z), int(n),
                                 float(h), _ptr(S), _ptr(Vx), _ptr(Vy), _ptr(Vz), _ptr(nbr),
                                 int(out_order), _stream(stream)), "pi_submit_host")


def pi_submit_host_strided(ctx, lo, hi, r_c: float, x, y, z, in_stride: int, n: int, h: float, S, Vx, Vy, Vz,
                           nbr=None, out_stride: int = 0, out_order: int = PI_ORDER_ORIGINAL, stream=None) -> None:
    """pi_submit_host with host arrays that may lie in blocks (one copy per
    block); see include/pi.h."""
    box = PiBox((ctypes.c_float * 3)(*lo), (ctypes.c_float * 3)(*hi))
    _check(load().pi_submit_host_strided(ctx, ctypes.byref(box), float(r_c), _ptr(x), _ptr(y), _ptr(z),
                                         int(in_stride), int(n), float(h), _ptr(S), _ptr(Vx), _ptr(Vy),
                                         _ptr(Vz), _ptr(nbr), int(out_stride), int(out_order), _stream(stream)),
           "pi_submit_host_strided")


def pi_server_slot_bytes(capacity: int) -> int:
    return int(load().pi_server_slot_bytes(int(capacity)))


def pi_server_create(capacities, initial_slots=None, max_slots_per_bucket: int = 8, hbm_budget: int = 0):
    k = len(capacities)
    caps = (ctypes.c_int64 * k)(*[int(c) for c in capacities])
    init = (ctypes.c_int32 * k)(*[int(c) for c in initial_slots]) if initial_slots is not None else None
    out = ctypes.c_void_p()
    _check(load().pi_server_create(int(k), caps, init, int(max_slots_per_bucket), int(hbm_budget),
                                   ctypes.byref(out)), "pi_server_create")
    return Handle(out.value, "server")


def pi_server_run(srv, jobs) -> float:
    """Serves a ctypes array of PiJob; returns the makespan in seconds."""
    mk = ctypes.c_double()
    _check(load().pi_server_run(srv, jobs, len(jobs), ctypes.byref(mk)), "pi_server_run")
    return mk.value


def pi_server_info(srv):
    """(capacities, slots per bucket, bytes charged to the HBM budget)."""
    nb = ctypes.c_int32()
    caps = (ctypes.c_int64 * PI_SERVER_MAX_BUCKETS)()
    slots = (ctypes.c_int32 * PI_SERVER_MAX_BUCKETS)()
    used = ctypes.c_int64()
    _check(load().pi_server_info(srv, ctypes.byref(nb), caps, slots, ctypes.byref(used)), "pi_server_info")
    return list(caps[: nb.value]), list(slots[: nb.value]), used.value


def pi_server_destroy(srv) -> None:
    _check(load().pi_server_destroy(srv), "pi_server_destroy")
    if isinstance(srv, Handle):
        srv._close()


def pi_grid(ctx):
    dims = (ctypes.c_int32 * 3)()
    _check(load().pi_grid(ctx, ctypes.cast(dims, ctypes.c_void_p)), "pi_grid")
    return tuple(dims)


def pi_binned(ctx) -> dict:
    ptrs = [ctypes.c_void_p() for _ in range(6)]
    _check(load().pi_binned(ctx, *[ctypes.byref(p) for p in ptrs]), "pi_binned")
    names = ("counts", "offsets", "perm", "sx", "sy", "sz")
    return {k: p.value for k, p in zip(names, ptrs)}


def pi_copy_binned(ctx, counts=None, offsets=None, perm=None, sx=None, sy=None, sz=None,
                   stream=None) -> None:
    _check(load().pi_copy_binned(ctx, _ptr(counts), _ptr(offsets), _ptr(perm), _ptr(sx), _ptr(sy),
                                 _ptr(sz), _stream(stream)), "pi_copy_binned")


def _check_u32_device(t, need: int, what: str) -> None:
    """A contiguous tensor of 4-byte elements on the current CUDA device with
    at least ``need`` entries (checked before the C call, so that a short or
    foreign buffer never reaches a kernel)."""
    import torch

    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{what}: a torch tensor is required")
    if t.element_size() != 4 or t.is_floating_point() or t.is_complex():
        raise TypeError(f"{what}: 4-byte integer elements are required, not {t.dtype}")
    if not t.is_cuda or t.device.index != torch.cuda.current_device():
        raise ValueError(f"{what}: must be on the current CUDA device")
    if not t.is_contiguous():
        raise ValueError(f"{what}: must be contiguous")
    if t.numel() < need:
        raise ValueError(f"{what}: {t.numel()} entries, {need} needed")


def pi_scan_counts_noalloc(counts, C: int, offsets, result=None, stream=None) -> None:
    """Exclusive scan of C device counts into C+1 device offsets using the
    library's fixed scratch array (no allocation); result (2 uint32, device)
    receives M_C and the device error bits.  The tensors are checked here
    (4-byte integer elements, contiguous, on the current device, long
    enough); the library checks the size limit and the 16-byte alignment."""
    C = int(C)
    if C >= 1:
        _check_u32_device(counts, C, "counts")
        _check_u32_device(offsets, C + 1, "offsets")
        if result is not None:
            _check_u32_device(result, 2, "result")
    _check(load().pi_scan_counts_noalloc(_ptr(counts), C, _ptr(offsets), _ptr(result),
                                         _stream(stream)), "pi_scan_counts_noalloc")


def pi_autotune(ctx, h, S, Vx, Vy, Vz, nbr=None, out_order: int = PI_ORDER_SORTED, reps: int = 3,
                stream=None):
    """Times every tile shape, PI_ALGO_PPNL and (batches) a shape per
    occupancy regime on the binned data, keeps the fastest.  Returns (chosen
    index: shape 0..6, PI_AUTOTUNE_PPNL or PI_AUTOTUNE_REGIMES, [median ms
    per candidate])."""
    arr = (ctypes.c_float * len(h))(*[float(v) for v in h])
    chosen = ctypes.c_int32()
    ms = (ctypes.c_float * (PI_NUM_TILES + 2))()
    _check(load().pi_autotune(ctx, ctypes.cast(arr, ctypes.c_void_p), _ptr(S), _ptr(Vx), _ptr(Vy),
                              _ptr(Vz), _ptr(nbr), int(out_order), int(reps), ctypes.byref(chosen),
                              ctypes.cast(ms, ctypes.c_void_p), _stream(stream)), "pi_autotune")
    return chosen.value, list(ms)


def pi_total_f64(ctx, v, out, stream=None) -> None:
    """FP64 total of device array v over each system's particles into out
    (device float64, one entry per system)."""
    _check(load().pi_total_f64(ctx, _ptr(v), _ptr(out), _stream(stream)), "pi_total_f64")


def pi_sync_status(ctx, stream=None, raise_on_error: bool = True):
    """Synchronises and returns (status, max_per_cell)."""
    m = ctypes.c_uint32()
    st = load().pi_sync_status(ctx, _stream(stream), ctypes.byref(m))
    if raise_on_error:
        _check(st, "pi_sync_status")
    return st, int(m.value)


def pi_set_option(ctx, key: int, value: int) -> None:
    _check(load().pi_set_option(ctx, int(key), int(value)), "pi_set_option")


def pi_launch_count(ctx) -> int:
    c = ctypes.c_uint64()
    _check(load().pi_launch_count(ctx, ctypes.byref(c)), "pi_launch_count")
    return int(c.value)


def pi_eval_count(ctx, stream=None) -> int:
    """Synchronises and returns the target-source evaluations the direct
    kernels counted since the last bin (PI_OPT_COUNT_EVALS)."""
    c = ctypes.c_uint64()
    _check(load().pi_eval_count(ctx, _stream(stream), ctypes.byref(c)), "pi_eval_count")
    return int(c.value)

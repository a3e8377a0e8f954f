"""Helpers for the GPU parity tests: run one step through the C ABI and
compare it with the oracle element by element.

The GPU side is called only through ``paper_2406_16091_gb300.binding`` (the
C ABI); the expected values come only from ``oracle``.
"""
from __future__ import annotations

import numpy as np

import oracle
from paper_2406_16091_gb300 import binding as B

# Tolerance of the floating-point sums: |gpu - oracle| <= TOL * sum_j |term_j|
# per particle and output, with the sum of |terms| taken in FP64 by the oracle;
# where that sum is 0 the GPU value must be exactly 0.  The terms are FP32,
# and a Gaussian term below the smallest normal FP32 number (2^-126) is zero
# on the GPU (flush to zero): given the cutoff r_c, the check adds that much
# per neighbour (r_c times that for V, |d_ij| < r_c), which only matters for
# sums that small.
TOL = 1e-5
FTZ = 2.0 ** -126


def torch_mod():
    import torch
    return torch


def run_gpu(x, y, z, lo, hi, rc, h, algo=B.PI_ALGO_TILED, precision=B.PI_PREC_FP32,
            order=B.PI_ORDER_SORTED, n_max=None, binned=True, nbr=True, repeat=1,
            kernel=B.PI_KERNEL_GAUSSIAN, tile=None, binning=None):
    """One pi_bin + pi_interact on cuda:0.  Returns a dict of numpy arrays.
    binning: PI_BIN_PER_PARTICLE (the default), PI_BIN_BUCKETED or PI_BIN_RADIX."""
    torch = torch_mod()
    dev = torch.device("cuda", 0)
    n = len(x)
    ctx = B.pi_create(lo, hi, rc, n if n_max is None else n_max)
    try:
        B.pi_set_option(ctx, B.PI_OPT_ALGO, algo)
        B.pi_set_option(ctx, B.PI_OPT_PRECISION, precision)
        B.pi_set_option(ctx, B.PI_OPT_KERNEL, kernel)
        if tile is not None:
            B.pi_set_option(ctx, B.PI_OPT_TILE, tile)
        if binning is not None:
            B.pi_set_option(ctx, B.PI_OPT_BINNING, binning)
        s = torch.cuda.current_stream()
        tx, ty, tz = (torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(dev) for a in (x, y, z))
        m = max(n, 1)
        S, Vx, Vy, Vz = (torch.full((m,), float("nan"), device=dev) for _ in range(4))
        nb = torch.full((m,), -1, dtype=torch.int32, device=dev) if nbr else None
        for _ in range(repeat):
            B.pi_bin(ctx, tx, ty, tz, n, s)
            B.pi_interact(ctx, h, S, Vx, Vy, Vz, nb, order, s)
        out = {}
        if binned:
            dims = B.pi_grid(ctx)
            C = dims[0] * dims[1] * dims[2]
            counts = torch.empty(C, dtype=torch.int32, device=dev)
            offsets = torch.empty(C + 1, dtype=torch.int32, device=dev)
            perm = torch.empty(m, dtype=torch.int32, device=dev)
            sx, sy, sz = (torch.empty(m, device=dev) for _ in range(3))
            B.pi_copy_binned(ctx, counts, offsets, perm, sx, sy, sz, s)
            out.update(dims=dims, counts=counts, offsets=offsets, perm=perm[:n], sx=sx[:n],
                       sy=sy[:n], sz=sz[:n])
        st, mpc = B.pi_sync_status(ctx, s, raise_on_error=False)
        out.update(S=S[:n], Vx=Vx[:n], Vy=Vy[:n], Vz=Vz[:n])
        if nbr:
            out["nbr"] = nb[:n]
        res = {}
        for k, v in out.items():
            if hasattr(v, "cpu"):
                a = v.cpu().numpy()
                res[k] = a.view(np.uint32) if a.dtype == np.int32 else a
            else:
                res[k] = v
        res["status"] = st
        res["max_per_cell"] = mpc
        res["launches"] = B.pi_launch_count(ctx)
        return res
    finally:
        B.pi_destroy(ctx)


def oracle_run(x, y, z, lo, hi, rc, h, kernel=0):
    b = oracle.bin_particles(x, y, z, lo, hi, rc)
    r = oracle.interact(b, rc, h, kernel)
    return b, r


def check_binning(g, b):
    assert g["status"] == B.PI_OK, B.status_str(g["status"])
    assert tuple(g["dims"]) == tuple(b.dims)
    assert np.array_equal(g["counts"], b.counts)
    assert np.array_equal(g["offsets"], b.offsets)
    assert np.array_equal(g["perm"], b.perm)
    assert np.array_equal(g["sx"].view(np.uint32), b.sx.view(np.uint32))
    assert np.array_equal(g["sy"].view(np.uint32), b.sy.view(np.uint32))
    assert np.array_equal(g["sz"].view(np.uint32), b.sz.view(np.uint32))
    assert g["max_per_cell"] == b.max_per_cell


def sum_errors(g, r, perm=None, rc=None):
    """Largest |gpu - oracle| / sum|terms| per output (less the FP32
    underflow allowance when the cutoff rc is given); asserts exact zeros."""
    worst = {}
    for name, ref, ab in (("S", r.S, r.absS), ("Vx", r.Vx, r.absVx), ("Vy", r.Vy, r.absVy),
                          ("Vz", r.Vz, r.absVz)):
        got = g[name].astype(np.float64)
        if perm is not None:
            got = got[perm]
        zero = ab == 0
        assert np.all(got[zero] == 0.0), f"{name}: nonzero where no pair contributes"
        nz = ~zero
        err = np.abs(got[nz] - ref[nz])
        if rc is not None:
            floor = r.nbr[nz].astype(np.float64) * FTZ * (1.0 if name == "S" else float(rc))
            err = np.maximum(err - floor, 0.0)
        rel = err / ab[nz] if nz.any() else np.zeros(0)
        assert np.all(np.isfinite(got)), name
        worst[name] = float(rel.max()) if rel.size else 0.0
    return worst


def check_interaction(g, r, tol=TOL, perm=None, rc=None):
    """perm: for outputs in input order, the oracle's sorted-slot -> input map;
    rc: the cutoff, for the FP32 underflow allowance of short kernels."""
    nbr = g["nbr"] if perm is None else g["nbr"][perm]
    bad = np.nonzero(nbr != r.nbr)[0]
    assert bad.size == 0, f"neighbour counts differ at {bad[:10]}: {nbr[bad[:10]]} vs {r.nbr[bad[:10]]}"
    worst = sum_errors(g, r, perm, rc)
    for k, v in worst.items():
        assert v <= tol, f"{k}: max relative error {v:.3e} > {tol:.0e}"
    return worst

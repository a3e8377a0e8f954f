"""GPU parity: every output of the CUDA path against the oracle, element by
element, on seeded inputs.

Bit-exact: counts, offsets, M_C, the stable permutation, the sorted
positions and the neighbour counts.  Within 1e-5 of sum|terms| per particle:
S, Vx, Vy, Vz.  Sizes run from empty and ragged inputs through several tiles
of every kernel to the full benchmark workloads, in the launch configuration
the benchmark times.
"""
import numpy as np

import oracle
import pytest

from paper_2406_16091_gb300 import binding as B
from paper_2406_16091_gb300 import workloads as W

from gpu_harness import check_binning, check_interaction, oracle_run, run_gpu

pytestmark = pytest.mark.gpu

ALGOS = [B.PI_ALGO_TILED, B.PI_ALGO_PPNL]
# (algorithm, tile shape): the one-CTA-per-chunk shapes of 32 and 128
# threads, both warp-specialised shapes, the direct form, and Alg. 1
VARIANTS = [(B.PI_ALGO_TILED, 0), (B.PI_ALGO_TILED, 2), (B.PI_ALGO_TILED, 3), (B.PI_ALGO_TILED, 4),
            (B.PI_ALGO_TILED, 5), (B.PI_ALGO_TILED, 6), (B.PI_ALGO_PPNL, None)]
VARIANT_IDS = ["tile0", "tile2", "ws4", "ws8", "direct", "direct4", "ppnl"]


def _case(w):
    x, y, z = w.positions()
    return x, y, z, w.lo, w.hi, w.rc, w.h


SMALL_CASES = {
    "small": W.SMALL,
    "ragged_4099": W.scaled(W.SMALL, 4099),
    "ragged_1023_ppc1": W.scaled(W.SCALE_VARIANTS[1], 1023),
    "ppc32_20000": W.scaled(W.SCALE_VARIANTS[32], 20000),
    "clustered_60000": W.scaled(W.CLUSTERED, 60000),
}


@pytest.mark.parametrize("name", list(SMALL_CASES))
@pytest.mark.parametrize("variant", VARIANTS, ids=VARIANT_IDS)
def test_small_workloads(name, variant):
    x, y, z, lo, hi, rc, h = _case(SMALL_CASES[name])
    b, r = oracle_run(x, y, z, lo, hi, rc, h)
    algo, tile = variant
    g = run_gpu(x, y, z, lo, hi, rc, h, algo=algo, tile=tile)
    check_binning(g, b)
    check_interaction(g, r)


@pytest.mark.parametrize("n", [0, 1, 2, 3, 5, 31, 33, 127, 4097])
def test_tiny_and_ragged_sizes(n):
    x, y, z = W.uniform(n, 100 + n)
    rc = 0.2
    b, r = oracle_run(x, y, z, (0, 0, 0), (1, 1, 1), rc, rc / 2)
    for algo, tile in VARIANTS:
        g = run_gpu(x, y, z, (0, 0, 0), (1, 1, 1), rc, rc / 2, algo=algo, tile=tile, n_max=n + 7)
        check_binning(g, b)
        if n:
            check_interaction(g, r)


def test_non_cubic_box_with_offset():
    lo, hi = (-1.0, 0.5, 2.0), (1.0, 1.5, 2.25)
    x, y, z = W.uniform(30000, 77, lo, hi)
    rc = 0.031
    b, r = oracle_run(x, y, z, lo, hi, rc, rc / 2)
    for algo, tile in VARIANTS:
        g = run_gpu(x, y, z, lo, hi, rc, rc / 2, algo=algo, tile=tile)
        check_binning(g, b)
        check_interaction(g, r)


def test_long_rows_longer_than_a_chunk():
    """300 cells along X, few per cell: X-rows are split into several chunks."""
    lo, hi = (0.0, 0.0, 0.0), (3.0, 0.04, 0.04)
    x, y, z = W.uniform(3000, 5, lo, hi)
    rc = 0.01
    b, r = oracle_run(x, y, z, lo, hi, rc, rc / 2)
    assert b.dims[0] == 300
    for algo, tile in VARIANTS:
        g = run_gpu(x, y, z, lo, hi, rc, rc / 2, algo=algo, tile=tile)
        check_binning(g, b)
        check_interaction(g, r)


def test_dense_cell_overflows_shared_memory():
    """A cluster whose neighbour rows hold more particles than one staged
    chunk fits: that chunk is read from global memory instead."""
    rng = np.random.default_rng(3)
    bg = rng.random((20000, 3)).astype(np.float32)
    cl = (0.5 + 0.004 * rng.standard_normal((6000, 3))).astype(np.float32)
    p = np.concatenate([bg, cl])
    rc = 1.0 / 64
    b, r = oracle_run(p[:, 0], p[:, 1], p[:, 2], (0, 0, 0), (1, 1, 1), rc, rc / 2)
    assert b.max_per_cell > 300
    for algo, tile in VARIANTS:
        g = run_gpu(p[:, 0], p[:, 1], p[:, 2], (0, 0, 0), (1, 1, 1), rc, rc / 2, algo=algo, tile=tile)
        check_binning(g, b)
        check_interaction(g, r)


def test_lattice_on_cell_faces():
    """Dyadic lattice points sitting exactly on cell faces, spacing = r_c:
    every axis neighbour is exactly r_c away and must not count."""
    m = 32
    g1 = (np.arange(m) / m).astype(np.float32)
    X, Y, Z = np.meshgrid(g1, g1, g1, indexing="ij")
    x, y, z = X.ravel(), Y.ravel(), Z.ravel()
    rc = 1.0 / m
    b, r = oracle_run(x, y, z, (0, 0, 0), (1, 1, 1), rc, rc / 2)
    assert r.nbr.max() == 0
    for algo, tile in VARIANTS:
        g = run_gpu(x, y, z, (0, 0, 0), (1, 1, 1), rc, rc / 2, algo=algo, tile=tile)
        check_binning(g, b)
        check_interaction(g, r)
    rc2 = 1.5 / m
    b, r = oracle_run(x, y, z, (0, 0, 0), (1, 1, 1), rc2, rc2 / 2)
    for algo, tile in VARIANTS:
        g = run_gpu(x, y, z, (0, 0, 0), (1, 1, 1), rc2, rc2 / 2, algo=algo, tile=tile)
        check_binning(g, b)
        check_interaction(g, r)


@pytest.mark.parametrize("box,rc,n", [
    (((0, 0, 0), (1, 1, 1)), 1.5, 600),            # one cell: every pair a candidate
    (((0, 0, 0), (1, 1, 1)), 0.5, 800),            # 2 x 2 x 2 cells, all at a boundary
    (((0, 0, 0), (4, 0.3, 0.3)), 0.31, 700),       # cells only along X (rows of 12 cells)
    (((0, 0, 0), (0.3, 0.3, 4)), 0.31, 700),       # one cell per X-row, a stack along Z
    (((0, 0, 0), (0.3, 4, 0.3)), 0.31, 700),       # one cell per X-row, a stack along Y
])
def test_degenerate_grids(box, rc, n):
    """Grids with one cell per axis or per row: windows clip to the single
    row, every X-row is one cell followed by its sentinel slots."""
    lo, hi = box
    x, y, z = W.uniform(n, 31 + n, lo, hi)
    b, r = oracle_run(x, y, z, lo, hi, rc, rc / 2)
    for algo, tile in VARIANTS:
        g = run_gpu(x, y, z, lo, hi, rc, rc / 2, algo=algo, tile=tile)
        check_binning(g, b)
        check_interaction(g, r)


def _random_case(seed):
    """A seeded random configuration: box offset and extents, cutoff,
    particle count (empty and ragged included), layout and kernel width."""
    rng = np.random.default_rng(seed)
    lo = tuple(float(v) for v in rng.uniform(-3, 3, 3).astype(np.float32))
    ext = rng.uniform(0.2, 3.0, 3)
    hi = tuple(float(np.float32(l + e)) for l, e in zip(lo, ext))
    cells = rng.integers(1, 24, 3)
    rc = float(np.float32(min(e / c for e, c in zip(ext, cells)) * rng.uniform(0.6, 1.0)))
    n = int(rng.choice([0, 1, 33, 500, 3000, 12000, 30000, 60000]))
    if n >= 500 and rng.random() < 0.5:
        x, y, z = W.clustered(n, 500 + seed)
        x, y, z = (np.float32(l) + np.float32(e) * a for l, e, a in zip(lo, ext, (x, y, z)))
        x, y, z = (np.minimum(a.astype(np.float32), np.nextafter(np.float32(h), np.float32(l))).astype(np.float32)
                   for a, l, h in zip((x, y, z), lo, hi))
    else:
        x, y, z = W.uniform(n, 500 + seed, lo, hi)
    h = float(rc * rng.uniform(0.1, 1.2))
    return x, y, z, lo, hi, rc, h


@pytest.mark.parametrize("seed", range(24))
def test_random_configurations(seed):
    """Seeded random boxes, cutoffs, sizes and layouts through the direct
    kernel (both precision modes), a staged shape and Alg. 1."""
    x, y, z, lo, hi, rc, h = _random_case(seed)
    b, r = oracle_run(x, y, z, lo, hi, rc, h)
    for algo, tile, prec in ((B.PI_ALGO_TILED, 5, B.PI_PREC_FP32), (B.PI_ALGO_TILED, 5, B.PI_PREC_KAHAN),
                             (B.PI_ALGO_TILED, 6, B.PI_PREC_FP32), (B.PI_ALGO_TILED, 2, B.PI_PREC_FP32),
                             (B.PI_ALGO_PPNL, None, B.PI_PREC_FP32)):
        g = run_gpu(x, y, z, lo, hi, rc, h, algo=algo, tile=tile, precision=prec, n_max=max(len(x), 1))
        check_binning(g, b)
        if len(x):
            check_interaction(g, r, rc=rc)


# Short kernels (h a small fraction of r_c): every path excludes the self
# pair by identity, so a particle's sum is never rounded at the size of
# K(0) = 1; from r_c^2/h^2 > 16 on the Gaussian's exponent is compensated
# (at h = r_c/4 the plain FP32 form runs, at r_c/8 and r_c/12 the fine one).
SHORT_VARIANTS = [(B.PI_ALGO_TILED, 0, B.PI_PREC_FP32), (B.PI_ALGO_TILED, 2, B.PI_PREC_FP32),
                  (B.PI_ALGO_TILED, 5, B.PI_PREC_FP32), (B.PI_ALGO_TILED, 6, B.PI_PREC_FP32),
                  (B.PI_ALGO_PPNL, None, B.PI_PREC_FP32), (B.PI_ALGO_TILED, 5, B.PI_PREC_KAHAN),
                  (B.PI_ALGO_TILED, 6, B.PI_PREC_KAHAN)]
SHORT_CASES = {
    "scale_ppc1": W.SCALE_VARIANTS[1],
    "clustered_400000": W.scaled(W.CLUSTERED, 400000),
}


@pytest.mark.parametrize("hdiv", [4, 8])
@pytest.mark.parametrize("name", list(SHORT_CASES))
def test_short_kernel_lengths(name, hdiv):
    w = SHORT_CASES[name]
    x, y, z = w.positions()
    h = w.rc / hdiv
    b, r = oracle_run(x, y, z, w.lo, w.hi, w.rc, h)
    for algo, tile, prec in SHORT_VARIANTS:
        g = run_gpu(x, y, z, w.lo, w.hi, w.rc, h, algo=algo, tile=tile, precision=prec)
        check_binning(g, b)
        check_interaction(g, r, rc=w.rc)


@pytest.mark.parametrize("hdiv", [2, 4, 8, 12])
def test_two_particles_near_the_cutoff(hdiv):
    """Two particles 0.9 r_c apart: each sees the other alone, S = exp(-0.81
    (r_c/h)^2) -- at h = r_c/12 below 2^-126, where FP32 flushes it to 0."""
    rng = np.random.default_rng(hdiv)
    rc = 1.0 / 16
    for k in range(8):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        p0 = rng.uniform(0.2, 0.8, 3)
        p1 = p0 + 0.9 * rc * u
        x, y, z = (np.array([p0[i], p1[i]], np.float32) for i in range(3))
        h = rc / hdiv
        b, r = oracle_run(x, y, z, (0, 0, 0), (1, 1, 1), rc, h)
        assert r.nbr.tolist() == [1, 1]
        for algo, tile, prec in SHORT_VARIANTS:
            g = run_gpu(x, y, z, (0, 0, 0), (1, 1, 1), rc, h, algo=algo, tile=tile, precision=prec)
            check_binning(g, b)
            check_interaction(g, r, rc=rc)
            if hdiv <= 8:
                assert np.all(g["S"] > 0)


def test_kernel_length_without_fp32_scale_is_rejected():
    """h so small that -log2(e)/h^2 overflows FP32: refused on the host."""
    x, y, z = W.uniform(100, 3)
    with pytest.raises(B.PiError) as e:
        run_gpu(x, y, z, (0, 0, 0), (1, 1, 1), 0.1, 1e-20)
    assert e.value.status == B.PI_ERR_INVALID_ARG
    assert "finite FP32 kernel scale" in B.last_error()


def test_coincident_particles():
    x = np.full(50, 0.3, np.float32)
    y = np.full(50, 0.6, np.float32)
    b, r = oracle_run(x, y, x, (0, 0, 0), (1, 1, 1), 0.1, 0.05)
    for algo, tile in VARIANTS:
        g = run_gpu(x, y, x, (0, 0, 0), (1, 1, 1), 0.1, 0.05, algo=algo, tile=tile)
        check_binning(g, b)
        check_interaction(g, r)
        assert np.all(g["S"] == 49.0)


def test_original_order_output():
    x, y, z, lo, hi, rc, h = _case(W.scaled(W.SMALL, 10000))
    b, r = oracle_run(x, y, z, lo, hi, rc, h)
    for algo, tile in VARIANTS:
        g = run_gpu(x, y, z, lo, hi, rc, h, algo=algo, tile=tile, order=B.PI_ORDER_ORIGINAL)
        check_interaction(g, r, perm=b.perm)


def test_kahan_precision_mode():
    """Compensated accumulation: same counts, and no larger error than the
    plain FP32 sums on a 32-per-cell workload."""
    x, y, z, lo, hi, rc, h = _case(W.scaled(W.SCALE_VARIANTS[32], 40000))
    b, r = oracle_run(x, y, z, lo, hi, rc, h)
    for algo, tile in VARIANTS:
        plain = check_interaction(run_gpu(x, y, z, lo, hi, rc, h, algo=algo, tile=tile), r)
        kahan = check_interaction(
            run_gpu(x, y, z, lo, hi, rc, h, algo=algo, tile=tile, precision=B.PI_PREC_KAHAN), r)
        assert kahan["S"] <= plain["S"] * 1.01 + 1e-9


def test_repeat_is_deterministic():
    x, y, z, lo, hi, rc, h = _case(W.scaled(W.CLUSTERED, 50000))
    a = run_gpu(x, y, z, lo, hi, rc, h, repeat=1, tile=3)
    c = run_gpu(x, y, z, lo, hi, rc, h, repeat=3, tile=3)
    for k in ("counts", "offsets", "perm", "sx", "nbr", "S", "Vx", "Vy", "Vz"):
        assert np.array_equal(a[k].view(np.uint32), c[k].view(np.uint32)), k


# ---- full-size workloads, in the launch configuration bench.py times -------------

FULL = ["small", "scale", "scale_ppc1", "scale_ppc2", "scale_ppc4", "scale_ppc16",
        "scale_ppc32", "clustered"]


@pytest.mark.parametrize("name", FULL)
def test_full_size_workloads(name):
    w = W.WORKLOADS[name]
    x, y, z, lo, hi, rc, h = _case(w)
    b, r = oracle_run(x, y, z, lo, hi, rc, h)
    g = run_gpu(x, y, z, lo, hi, rc, h)
    check_binning(g, b)
    check_interaction(g, r)
    # each within-cutoff pair is seen from both sides
    assert int(g["nbr"].astype(np.int64).sum()) % 2 == 0


def test_full_size_precision_and_comparator_rows():
    """At full size in the bench's launch configuration: the compensated
    sums on the 4.2 M clustered workload (the precision row) and the
    Lennard-Jones comparator on the 2 M scale workload match the oracle, and
    the compensated error is no larger than the plain one."""
    w = W.WORKLOADS["clustered"]
    x, y, z, lo, hi, rc, h = _case(w)
    b, r = oracle_run(x, y, z, lo, hi, rc, h)
    plain = check_interaction(run_gpu(x, y, z, lo, hi, rc, h, binned=False), r)
    kahan = check_interaction(run_gpu(x, y, z, lo, hi, rc, h, precision=B.PI_PREC_KAHAN, binned=False), r)
    assert kahan["S"] <= plain["S"]
    w = W.WORKLOADS["scale"]
    x, y, z, lo, hi, rc, h = _case(w)
    b, r = oracle_run(x, y, z, lo, hi, rc, h, oracle.LJ)
    check_interaction(run_gpu(x, y, z, lo, hi, rc, h, kernel=B.PI_KERNEL_LJ, binned=False), r)


def test_large_system_64m_particles():
    """2^26 particles on a 203^3 grid (8 per cell, 8.4 M cells, about 5 GB on
    the device): particle indices, offsets and P slots past 2^26, every
    output against the oracle."""
    w = W.scaled(W.SCALE, 1 << 26)
    assert w.cells_per_axis() == 203
    x, y, z, lo, hi, rc, h = _case(w)
    b, r = oracle_run(x, y, z, lo, hi, rc, h)
    g = run_gpu(x, y, z, lo, hi, rc, h)
    check_binning(g, b)
    check_interaction(g, r)


# ---- failure paths: no fault, the status comes back and the context recovers ----

def test_out_of_box_reported_then_recovers():
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    x, y, z = W.uniform(5000, 9)
    bad = x.copy()
    bad[1234] = 1.5
    ctx = B.pi_create((0, 0, 0), (1, 1, 1), 0.1, 5000)
    try:
        s = torch.cuda.current_stream()
        tb, ty, tz = (torch.from_numpy(a).to(dev) for a in (bad, y, z))
        out = [torch.empty(5000, device=dev) for _ in range(4)]
        B.pi_bin(ctx, tb, ty, tz, 5000, s)
        B.pi_interact(ctx, 0.05, *out, None, B.PI_ORDER_SORTED, s)
        st, _ = B.pi_sync_status(ctx, s, raise_on_error=False)
        assert st == B.PI_ERR_OUT_OF_BOX
        tx = torch.from_numpy(x).to(dev)
        B.pi_bin(ctx, tx, ty, tz, 5000, s)
        B.pi_interact(ctx, 0.05, *out, None, B.PI_ORDER_SORTED, s)
        st, _ = B.pi_sync_status(ctx, s, raise_on_error=False)
        assert st == B.PI_OK
        with pytest.raises(B.PiError) as e:
            B.pi_bin(ctx, tx, ty, tz, 5001, s)
        assert e.value.status == B.PI_ERR_CAPACITY
    finally:
        B.pi_destroy(ctx)


def test_scan_wait_times_out_and_recovers():
    """The first scan tile withholds its prefix (a flag nothing sets): the
    other tiles' bounded waits run out, the status is PI_ERR_TIMEOUT, and the
    next step succeeds."""
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    w = W.scaled(W.SCALE, 200000)
    x, y, z = w.positions()
    ctx = B.pi_create(w.lo, w.hi, w.rc, w.n)
    try:
        dims = B.pi_grid(ctx)
        assert dims[0] * dims[1] * dims[2] > 4096  # at least two scan tiles
        s = torch.cuda.current_stream()
        tx, ty, tz = (torch.from_numpy(a).to(dev) for a in (x, y, z))
        out = [torch.empty(w.n, device=dev) for _ in range(4)]
        B.pi_set_option(ctx, B.PI_OPT_WAIT_LIMIT_NS, 20_000_000)
        B.pi_set_option(ctx, B.PI_OPT_TEST_WITHHOLD_SCAN, 1)
        B.pi_bin(ctx, tx, ty, tz, w.n, s)
        B.pi_interact(ctx, w.h, *out, None, B.PI_ORDER_SORTED, s)
        st, _ = B.pi_sync_status(ctx, s, raise_on_error=False)
        assert st == B.PI_ERR_TIMEOUT
        B.pi_set_option(ctx, B.PI_OPT_TEST_WITHHOLD_SCAN, 0)
        B.pi_bin(ctx, tx, ty, tz, w.n, s)
        B.pi_interact(ctx, w.h, *out, None, B.PI_ORDER_SORTED, s)
        st, mpc = B.pi_sync_status(ctx, s, raise_on_error=False)
        assert st == B.PI_OK and mpc > 0
    finally:
        B.pi_destroy(ctx)


def test_host_buffer_step_matches_device_step():
    torch = pytest.importorskip("torch")
    x, y, z, lo, hi, rc, h = _case(W.scaled(W.SMALL, 20000))
    b, r = oracle_run(x, y, z, lo, hi, rc, h)
    n = len(x)
    ctx = B.pi_create(lo, hi, rc, n)
    try:
        hx, hy, hz = (torch.from_numpy(a).pin_memory() for a in (x, y, z))
        outs = [torch.empty(n).pin_memory() for _ in range(4)]
        nb = torch.empty(n, dtype=torch.int32).pin_memory()
        B.pi_run_host(ctx, hx, hy, hz, n, h, *outs, nb, B.PI_ORDER_ORIGINAL,
                      torch.cuda.current_stream())
        g = {"S": outs[0].numpy(), "Vx": outs[1].numpy(), "Vy": outs[2].numpy(),
             "Vz": outs[3].numpy(), "nbr": nb.numpy().view(np.uint32)}
        check_interaction(g, r, perm=b.perm)
    finally:
        B.pi_destroy(ctx)

"""The three binning paths against each other and the oracle.

PI_BIN_PER_PARTICLE (the default) takes one global atomic and one provisional
record per particle; PI_BIN_BUCKETED counts the particles per bucket of
consecutive cells and ranks each bucket's cells in shared memory (buckets
too large for it go through a grid-wide path); PI_BIN_RADIX sorts the
particles by cell with a stable least-significant-digit radix sort (one,
two or three digit passes by the number of cells).  All must give the same counts, offsets,
M_C, stable permutation and sorted positions bit for bit (checked against
the oracle), and the same x-ordered copy and sub-bin words (checked through
the interaction's outputs, which read them, bitwise)."""
import numpy as np
import pytest

from paper_2406_16091_gb300 import binding as B
from paper_2406_16091_gb300 import workloads as W

from gpu_harness import check_binning, check_interaction, oracle_run, run_gpu

pytestmark = pytest.mark.gpu


def _dense_cluster(n_bg=20000, n_cl=6000, sigma=0.004, seed=3):
    rng = np.random.default_rng(seed)
    bg = rng.random((n_bg, 3)).astype(np.float32)
    cl = np.clip(0.5 + sigma * rng.standard_normal((n_cl, 3)), 0, np.nextafter(1, 0)).astype(np.float32)
    p = np.concatenate([bg, cl])
    return p[:, 0], p[:, 1], p[:, 2]


def _one_giant_cell():
    """6000 particles inside one cell (more than a bucket ranks in shared
    memory) in a sparse background."""
    rng = np.random.default_rng(11)
    bg = rng.random((3000, 3)).astype(np.float32)
    cell = (0.5 + (1.0 / 64) * rng.random((6000, 3)) * 0.9).astype(np.float32)
    p = np.concatenate([bg, cell])
    return p[:, 0], p[:, 1], p[:, 2]


def _workload(w):
    x, y, z = w.positions()
    return x, y, z, w.lo, w.hi, w.rc, w.h


CASES = {
    "small": lambda: _workload(W.SMALL),
    "ragged_4099": lambda: _workload(W.scaled(W.SMALL, 4099)),
    "ppc1_200000": lambda: _workload(W.scaled(W.SCALE_VARIANTS[1], 200000)),
    "ppc32_150000": lambda: _workload(W.scaled(W.SCALE_VARIANTS[32], 150000)),
    "clustered_500000": lambda: _workload(W.scaled(W.CLUSTERED, 500000)),
    "dense_cluster": lambda: (*_dense_cluster(), (0, 0, 0), (1, 1, 1), 1.0 / 64, 1.0 / 128),
    "one_giant_cell": lambda: (*_one_giant_cell(), (0, 0, 0), (1, 1, 1), 1.0 / 64, 1.0 / 128),
    "one_cell_grid": lambda: (*W.uniform(700, 5), (0, 0, 0), (1, 1, 1), 1.5, 0.75),
    "long_rows": lambda: (*W.uniform(5000, 6, (0, 0, 0), (3.0, 0.04, 0.04)), (0, 0, 0), (3.0, 0.04, 0.04),
                          0.01, 0.005),
    # 81^3 = 531,441 cells: 20-bit keys, three radix passes of 7 bits
    "three_digit_passes": lambda: (*W.uniform(150000, 8), (0, 0, 0), (1, 1, 1), 1.0 / 81, 1.0 / 162),
    # 4^3 cells: one radix pass of 6 bits
    "one_digit_pass": lambda: (*W.uniform(30000, 9), (0, 0, 0), (1, 1, 1), 0.25, 0.125),
    # the bench's workload at full size (2,097,152 particles, 64^3 cells)
    "scale_full": lambda: _workload(W.SCALE),
}

PATHS = (B.PI_BIN_RADIX, B.PI_BIN_BUCKETED, B.PI_BIN_PER_PARTICLE)


@pytest.mark.parametrize("name", list(CASES))
def test_binning_paths_bitwise_equal(name):
    x, y, z, lo, hi, rc, h = CASES[name]()
    b, r = oracle_run(x, y, z, lo, hi, rc, h)
    got = {}
    for path in PATHS:
        for tile in (5, 6, 2):
            g = run_gpu(x, y, z, lo, hi, rc, h, tile=tile, binning=path)
            check_binning(g, b)
            check_interaction(g, r)
            got[(path, tile)] = g
    ref = got[(B.PI_BIN_PER_PARTICLE, 5)]
    for key, g in got.items():
        for k in ("counts", "offsets", "perm", "sx", "sy", "sz", "S", "Vx", "Vy", "Vz", "nbr"):
            assert np.array_equal(g[k].view(np.uint32), ref[k].view(np.uint32)), (key, k)


@pytest.mark.parametrize("path", [B.PI_BIN_BUCKETED, B.PI_BIN_RADIX], ids=["bucketed", "radix"])
def test_binning_repeats_and_recovers_after_an_error(path):
    """Steps after a failed step (a position outside the box) and repeated
    steps on one context give the oracle's results."""
    w = W.scaled(W.CLUSTERED, 300000)
    x, y, z = w.positions()
    b, r = oracle_run(x, y, z, w.lo, w.hi, w.rc, w.h)
    g = run_gpu(x, y, z, w.lo, w.hi, w.rc, w.h, repeat=3, binning=path)
    check_binning(g, b)
    check_interaction(g, r)
    bad = x.copy()
    bad[17] = np.float32(1.5)
    g = run_gpu(bad, y, z, w.lo, w.hi, w.rc, w.h, binning=path)
    assert g["status"] == B.PI_ERR_OUT_OF_BOX


@pytest.mark.parametrize("name,path,launches", [
    ("small", B.PI_BIN_PER_PARTICLE, 5),        # zero, hist, scan, scatter, stabilise
    ("small", B.PI_BIN_BUCKETED, 6),            # zero, count, scan, scatter, cells, big
    ("one_digit_pass", B.PI_BIN_RADIX, 6),      # zero, keys, scan, split, gather, rank
    ("small", B.PI_BIN_RADIX, 9),               # 2^12 cells: two digit passes
    ("three_digit_passes", B.PI_BIN_RADIX, 12),
])
def test_launch_count_per_binning_path(name, path, launches):
    """pi_launch_count (the bench's gpu_launches) adds exactly the kernels
    each binning path launches."""
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    x, y, z, lo, hi, rc, h = CASES[name]()
    s = torch.cuda.current_stream()
    ctx = B.pi_create(lo, hi, rc, len(x))
    try:
        B.pi_set_option(ctx, B.PI_OPT_BINNING, path)
        t = [torch.from_numpy(a).to(dev) for a in (x, y, z)]
        before = B.pi_launch_count(ctx)
        B.pi_bin(ctx, *t, len(x), s)
        assert B.pi_launch_count(ctx) - before == launches
        assert B.pi_sync_status(ctx, s)[0] == B.PI_OK
    finally:
        B.pi_destroy(ctx)

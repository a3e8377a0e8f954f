"""Pins for the oracle's binning (cell index, counts, scan, stable scatter).

Each test checks the oracle against something other than itself: the
paper's worked examples (tests/golden), a library routine the step reduces to
(numpy's cumulative sum, stable argsort, bincount), or positions whose cell is
known exactly.  CPU only.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2406_16091_gb300 import workloads as W


def test_fig1_grid_example(golden_dir):
    """Sec. 2, Fig. 1: counts [2,1,3,0,2,1] on a 3x2 grid give offsets
    [0,2,3,6,6,8,9] (C+1 entries, last = N, empty cell repeats its offset)."""
    g = json.load(open(os.path.join(golden_dir, "fig1_grid_example.json")))
    nx, ny, nz = g["grid_cells"]
    rng = np.random.default_rng(0)
    xs, ys, zs = [], [], []
    for c, k in enumerate(g["counts"]):
        cx, cy = c % nx, c // nx
        for _ in range(k):
            xs.append(cx + rng.uniform(0.05, 0.95))
            ys.append(cy + rng.uniform(0.05, 0.95))
            zs.append(rng.uniform(0.05, 0.95))
    b = oracle.bin_particles(xs, ys, zs, (0, 0, 0), (nx, ny, nz), 1.0)
    assert b.ok
    assert b.dims == (nx, ny, nz)
    assert b.counts.tolist() == g["counts"]
    assert b.offsets.tolist() == g["offsets"]
    assert b.max_per_cell == max(g["counts"])


def test_prefix_sum_example(golden_dir):
    """Sec. 6 worked example: eight ones scan to 1..8 (inclusive); our
    exclusive form is 0..8 with the total last."""
    g = json.load(open(os.path.join(golden_dir, "prefix_sum_example.json")))
    off = oracle.exclusive_scan(g["input"])
    assert off[1:].tolist() == g["inclusive_prefix"]
    assert off[0] == 0


@pytest.mark.parametrize("C", [1, 2, 7, 64, 1000, 4097])
def test_scan_matches_cumsum(C):
    rng = np.random.default_rng(C)
    counts = rng.integers(0, 5, C).astype(np.uint32)
    counts[rng.random(C) < 0.3] = 0
    off = oracle.exclusive_scan(counts)
    ref = np.concatenate([[0], np.cumsum(counts.astype(np.uint64))])
    assert np.array_equal(off.astype(np.uint64), ref)


def test_cell_index_known_cells():
    """Dyadic positions sit exactly in known cells: centres, lower faces,
    and the last float below hi (clamped into the last cell)."""
    n = 16
    rc = 1.0 / n
    lo, hi = (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)
    dims = oracle.grid_dims(lo, hi, rc)
    assert dims == (n, n, n)
    k = np.arange(n)
    centres = ((k + 0.5) / n).astype(np.float32)
    faces = (k / n).astype(np.float32)
    top = np.nextafter(np.float32(1.0), np.float32(0.0))
    for xs, expect in ((centres, k), (faces, k), (np.full(n, top, np.float32), np.full(n, n - 1))):
        z = np.zeros(n, np.float32)
        cell, ok = oracle.cell_index(xs, z, z, lo, hi, dims)
        assert ok
        assert np.array_equal(cell, expect)
        cell, ok = oracle.cell_index(z, xs, z, lo, hi, dims)
        assert np.array_equal(cell, expect * n)
        cell, ok = oracle.cell_index(z, z, xs, lo, hi, dims)
        assert np.array_equal(cell, expect * n * n)


def test_cell_index_out_of_box_flagged():
    lo, hi = (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)
    dims = oracle.grid_dims(lo, hi, 0.25)
    half = np.full(2, 0.5, np.float32)
    for bad in (1.0, -1e-7, np.nan, np.inf):
        x = np.array([0.5, bad], np.float32)
        _, ok = oracle.cell_index(x, half, half, lo, hi, dims)
        assert not ok


def test_grid_dims_rule():
    """Cells per axis = max(1, floor(L / r_c)) so that the width is >= r_c
    (Sec. 3); a cutoff larger than the box gives one cell."""
    assert oracle.grid_dims((0, 0, 0), (1, 1, 1), 1.0 / 64) == (64, 64, 64)
    assert oracle.grid_dims((-1, 0, 2), (1, 3, 2.5), 0.25) == (8, 12, 2)
    # fl32(0.3) is a little above 0.3, so 3 / r_c falls just short of 10
    assert oracle.grid_dims((-1, 0, 2), (1, 3, 2.5), 0.3) == (6, 9, 1)
    assert oracle.grid_dims((0, 0, 0), (1, 1, 1), 5.0) == (1, 1, 1)
    for cells in (128, 102, 81, 51, 40, 16, 64):
        rc = W.rc_for_cells(cells)
        assert oracle.grid_dims((0, 0, 0), (1, 1, 1), rc) == (cells,) * 3
    with pytest.raises(ValueError):
        oracle.grid_dims((0, 0, 0), (1, 1, 1), 0.0)
    with pytest.raises(ValueError):
        oracle.grid_dims((0, 0, 0), (0, 1, 1), 0.1)


@pytest.mark.parametrize("name,n", [("small", 32768), ("clustered", 20000)])
def test_binning_invariants(name, n):
    """Counts = bincount of the cell ids, offsets = their exclusive scan,
    perm = numpy's stable argsort of the cell ids (input order inside a cell),
    sorted positions = gathered positions, M_C = largest count."""
    w = W.WORKLOADS[name]
    if n != w.n:
        w = W.scaled(w, n)
    x, y, z = w.positions()
    b = oracle.bin_particles(x, y, z, w.lo, w.hi, w.rc)
    assert b.ok
    cell, ok = oracle.cell_index(x, y, z, w.lo, w.hi, b.dims)
    C = int(np.prod(b.dims))
    assert np.array_equal(b.counts, np.bincount(cell, minlength=C))
    assert b.offsets[-1] == n and b.offsets[0] == 0
    assert np.all(np.diff(b.offsets.astype(np.int64)) == b.counts)
    assert np.array_equal(b.perm, np.argsort(cell, kind="stable"))
    assert np.array_equal(np.sort(b.perm), np.arange(n))
    assert np.array_equal(b.sx, x[b.perm]) and np.array_equal(b.sy, y[b.perm])
    assert np.array_equal(b.sz, z[b.perm])
    assert b.max_per_cell == int(b.counts.max())


def test_binning_empty_and_single():
    b = oracle.bin_particles([], [], [], (0, 0, 0), (1, 1, 1), 0.25)
    assert b.ok and b.offsets.tolist() == [0] * 65 and b.max_per_cell == 0
    b = oracle.bin_particles([0.9], [0.1], [0.6], (0, 0, 0), (1, 1, 1), 0.25)
    assert b.perm.tolist() == [0]
    assert b.counts.argmax() == 3 + 4 * (0 + 4 * 2)

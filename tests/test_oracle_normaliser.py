"""Pins for the oracle's tolerance normaliser: the sums of |term| per output.

Every GPU parity check allows |gpu - oracle| <= 1e-5 * sum_j |term_j|, so the
normaliser absS = sum_j |K_ij| and absV_d = sum_j |d_ij,d| |K_ij| (d_ij =
p_j - p_i, Sec. 2's terms) must be right on its own: a factor on one output
or a lost absolute value would silently loosen or tighten every GPU test.
Each output is checked against closed forms -- a single Gaussian pair (both
sides, so each axis sees a negative offset), a dyadic lattice, the h -> inf
limit, a single Lennard-Jones pair with its two-term magnitude -- and against
the identities |S| <= absS, |V_d| <= absV_d with equality when every term has
one sign.  CPU only.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2406_16091_gb300 import workloads as W


def run(x, y, z, lo, hi, rc, h, kernel=oracle.GAUSSIAN):
    b = oracle.bin_particles(x, y, z, lo, hi, rc)
    assert b.ok
    r = oracle.interact(b, rc, h, kernel)
    u = lambda a: oracle.unpermute(a, b.perm)
    return r, {k: u(getattr(r, k)) for k in ("S", "Vx", "Vy", "Vz", "nbr", "absS", "absVx", "absVy", "absVz")}


def test_single_gaussian_pair_normaliser():
    """absS = K and absV_d = |d_d| K on both sides of one pair; the offsets
    have mixed signs (and flip on the other side), so a lost |.| on any axis
    changes one of the eight checked values."""
    rc, h = 0.25, 0.125
    pi = np.array([0.30, 0.40, 0.50], np.float32)
    pj = np.array([0.40, 0.36, 0.375], np.float32)   # dx > 0, dy < 0, dz < 0
    d = pj.astype(np.float64) - pi.astype(np.float64)
    K = math.exp(-float(d @ d) / (h * h))
    _, o = run([pi[0], pj[0]], [pi[1], pj[1]], [pi[2], pj[2]], (0, 0, 0), (1, 1, 1), rc, h)
    assert o["nbr"].tolist() == [1, 1]
    for side in (0, 1):
        assert o["absS"][side] == pytest.approx(K, rel=1e-15)
        assert o["absVx"][side] == pytest.approx(abs(d[0]) * K, rel=1e-14)
        assert o["absVy"][side] == pytest.approx(abs(d[1]) * K, rel=1e-14)
        assert o["absVz"][side] == pytest.approx(abs(d[2]) * K, rel=1e-14)
    # equality with |S| and |V| here: one term per output
    assert np.allclose(o["absS"], np.abs(o["S"]), rtol=1e-15)
    for ax in ("x", "y", "z"):
        assert np.allclose(o["absV" + ax], np.abs(o["V" + ax]), rtol=1e-15)


def test_lattice_normaliser_closed_form():
    """Dyadic simple cubic lattice (spacing a, a < r_c < a sqrt 2): inside,
    V = 0 but absV_d = 2 a K on each axis and absS = 6 K; on a face (x = 0)
    absVx = a K while absVy = absVz = 2 a K."""
    m = 16
    a = 1.0 / m
    g = ((np.arange(m) + 0.5) / m).astype(np.float32)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    x, y, z = X.ravel(), Y.ravel(), Z.ravel()
    rc, h = 1.2 * a, 0.5 * a
    _, o = run(x, y, z, (0, 0, 0), (1, 1, 1), rc, h)
    ix, iy, iz = (np.rint(v * m - 0.5).astype(int) for v in (x, y, z))
    K = math.exp(-(a * a) / (h * h))
    inner = (ix > 0) & (ix < m - 1) & (iy > 0) & (iy < m - 1) & (iz > 0) & (iz < m - 1)
    assert np.allclose(o["absS"][inner], 6 * K, rtol=1e-14)
    for ax in ("absVx", "absVy", "absVz"):
        assert np.allclose(o[ax][inner], 2 * a * K, rtol=1e-14)
    face = (ix == 0) & (iy > 0) & (iy < m - 1) & (iz > 0) & (iz < m - 1)
    assert np.allclose(o["absVx"][face], a * K, rtol=1e-14)
    assert np.allclose(o["absVy"][face], 2 * a * K, rtol=1e-14)
    assert np.allclose(o["absVz"][face], 2 * a * K, rtol=1e-14)
    assert np.allclose(o["absS"][face], 5 * K, rtol=1e-14)


def test_wide_kernel_normaliser():
    """h -> inf gives K = 1: absS = n_i and absV_d = sum_j |p_j,d - p_i,d|
    over the n_i neighbours (found here by brute force)."""
    w = W.scaled(W.SMALL, 2500)
    x, y, z = w.positions()
    _, o = run(x, y, z, w.lo, w.hi, w.rc, 1e30)
    assert np.array_equal(o["absS"], o["nbr"].astype(np.float64))
    pos = np.stack([x, y, z], 1)
    rc2 = np.float32(w.rc) * np.float32(w.rc)
    rng = np.random.default_rng(17)
    for i in rng.choice(len(x), 60, replace=False):
        d32 = (pos - pos[i]).astype(np.float32)
        # the FP32 predicate: dx*dx rounded, then two fused steps (exact
        # products in FP64, one rounding to FP32 each)
        r2 = (d32[:, 0] * d32[:, 0]).astype(np.float32)
        r2 = (d32[:, 1].astype(np.float64) ** 2 + r2).astype(np.float32)
        r2 = (d32[:, 2].astype(np.float64) ** 2 + r2).astype(np.float32)
        if np.any(np.abs(r2.astype(np.float64) / float(rc2) - 1) < 1e-6):
            continue  # a candidate within rounding of the cutoff: skip this target
        js = np.nonzero(r2 < rc2)[0]
        js = js[js != i]
        assert len(js) == o["nbr"][i]
        dd = pos[js].astype(np.float64) - pos[i].astype(np.float64)
        for k, ax in enumerate(("absVx", "absVy", "absVz")):
            assert o[ax][i] == pytest.approx(np.abs(dd[:, k]).sum(), rel=1e-12, abs=1e-300)


def test_lennard_jones_pair_normaliser():
    """Lennard-Jones 4 (s^6 - s^3) cancels near its zero crossing, so the
    normaliser takes the two terms' magnitudes, 4 (s^6 + s^3); absV_d scales
    it by |d_d|."""
    sigma = float(np.float32(0.05))
    x = np.array([0.3, 0.33], np.float32)
    y = np.array([0.5, 0.49], np.float32)
    d = (float(x[1]) - float(x[0]), float(y[1]) - float(y[0]))
    r2 = d[0] ** 2 + d[1] ** 2
    s = sigma * sigma / (r2 + sigma * sigma / 100)
    mag = 4 * (s ** 6 + s ** 3)
    _, o = run(x, y, [0.5, 0.5], (0, 0, 0), (1, 1, 1), 0.2, sigma, oracle.LJ)
    for side in (0, 1):
        assert o["absS"][side] == pytest.approx(mag, rel=1e-12)
        assert o["absVx"][side] == pytest.approx(abs(d[0]) * mag, rel=1e-12)
        assert o["absVy"][side] == pytest.approx(abs(d[1]) * mag, rel=1e-12)
        assert o["absVz"][side] == 0.0


def test_normaliser_bounds_on_random_systems():
    """|S| <= absS and |V_d| <= absV_d for every particle, with equality for
    S (all Gaussian terms are positive); absV_d <= r_c absS per axis; and
    absS / n_i lies in [exp(-r_c^2/h^2), 1]."""
    for seed, (lo, hi, rc) in enumerate((((0, 0, 0), (1, 1, 1), 0.08),
                                         ((-1.0, 0.5, 2.0), (1.0, 1.5, 2.25), 0.11))):
        x, y, z = W.uniform(3000, 100 + seed, lo, hi)
        h = rc / 3
        _, o = run(x, y, z, lo, hi, rc, h)
        assert np.allclose(o["absS"], o["S"], rtol=1e-14, atol=0)
        for ax in ("x", "y", "z"):
            assert np.all(np.abs(o["V" + ax]) <= o["absV" + ax] * (1 + 1e-14))
            assert np.all(o["absV" + ax] <= rc * o["absS"] * (1 + 1e-12))
        has = o["nbr"] > 0
        per = o["absS"][has] / o["nbr"][has]
        assert np.all(per <= 1.0) and np.all(per >= math.exp(-(rc * rc) / (h * h)) * (1 - 1e-12))
        assert np.all(o["absS"][~has] == 0)

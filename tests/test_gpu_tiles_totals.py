"""Tile shapes and the autotuner give identical results; the FP64 totals
reproduce numpy's sums and show the vector-sum invariant (sum_i V_i = 0)."""
import numpy as np
import pytest

import oracle
from paper_2406_16091_gb300 import binding as B
from paper_2406_16091_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _setup(torch, w):
    dev = torch.device("cuda", 0)
    x, y, z = w.positions()
    ctx = B.pi_create(w.lo, w.hi, w.rc, w.n)
    s = torch.cuda.current_stream()
    t = [torch.from_numpy(a).to(dev) for a in (x, y, z)]
    out = [torch.empty(w.n, device=dev) for _ in range(4)]
    nb = torch.empty(w.n, dtype=torch.int32, device=dev)
    B.pi_bin(ctx, *t, w.n, s)
    return ctx, s, out, nb, (x, y, z)


@pytest.mark.parametrize("name", ["scale_ppc2", "small", "clustered"])
def test_tile_shapes_identical_and_autotune(name):
    torch = pytest.importorskip("torch")
    w = W.WORKLOADS[name]
    if w.n > 500000:
        w = W.scaled(w, 500000)
    ctx, s, out, nb, _ = _setup(torch, w)
    try:
        res = []
        for tile in range(B.PI_NUM_TILES):
            B.pi_set_option(ctx, B.PI_OPT_TILE, tile)
            B.pi_interact(ctx, w.h, *out, nb, B.PI_ORDER_SORTED, s)
            res.append([o.cpu().numpy().view(np.uint32).copy() for o in out + [nb]])
        for r in res[1:]:
            for a, b in zip(res[0], r):
                assert np.array_equal(a, b)
        chosen, ms = B.pi_autotune(ctx, [w.h], *out, nb, B.PI_ORDER_SORTED, 2, s)
        # shapes 0..6, Alg. 1, and the per-regime plan (batches only: 0 here)
        assert len(ms) == B.PI_NUM_TILES + 2 and ms[B.PI_AUTOTUNE_REGIMES] == 0
        ms = ms[:B.PI_NUM_TILES + 1]
        assert chosen in range(B.PI_NUM_TILES + 1) and all(m > 0 for m in ms)
        assert ms[chosen] == min(ms)
        # the chosen candidate stays in use
        B.pi_interact(ctx, w.h, *out, nb, B.PI_ORDER_SORTED, s)
        got = [o.cpu().numpy().view(np.uint32) for o in out + [nb]]
        if chosen < B.PI_NUM_TILES:
            for a, b in zip(res[0], got):
                assert np.array_equal(a, b)
        else:  # Alg. 1: same counts, sums within rounding
            assert np.array_equal(res[0][4], got[4])
            for a, b in zip(res[0][:4], got[:4]):
                fa, fb = a.view(np.float32), b.view(np.float32)
                assert np.allclose(fa, fb, rtol=1e-4, atol=1e-6)
        B.pi_sync_status(ctx, s)
    finally:
        B.pi_destroy(ctx)


def test_fp64_totals_and_vector_invariant():
    torch = pytest.importorskip("torch")
    w = W.scaled(W.CLUSTERED, 300000)
    ctx, s, out, nb, (x, y, z) = _setup(torch, w)
    try:
        B.pi_interact(ctx, w.h, *out, nb, B.PI_ORDER_SORTED, s)
        tot = torch.zeros(1, dtype=torch.float64, device="cuda")
        b = oracle.bin_particles(x, y, z, w.lo, w.hi, w.rc)
        r = oracle.interact(b, w.rc, w.h)
        for k, (o, ab) in enumerate(zip(out[1:], (r.absVx, r.absVy, r.absVz))):
            B.pi_total_f64(ctx, o, tot, s)
            got = float(tot.cpu()[0])
            host = o.cpu().numpy().astype(np.float64)
            assert got == pytest.approx(float(host.sum()), rel=1e-12, abs=1e-12 * float(np.abs(host).sum()))
            # each pair seen from both sides: the total vanishes up to FP32 rounding of the terms
            assert abs(got) <= 1e-5 * float(ab.sum())
        # deterministic: same bits on a second run
        B.pi_total_f64(ctx, out[1], tot, s)
        a1 = float(tot.cpu()[0])
        B.pi_total_f64(ctx, out[1], tot, s)
        assert float(tot.cpu()[0]) == a1
        B.pi_sync_status(ctx, s)
    finally:
        B.pi_destroy(ctx)


def test_fp64_totals_per_system_of_a_batch():
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    ns = [1000, 0, 25000, 7]
    boxes = [((0, 0, 0), (1, 1, 1))] * 4
    ctx = B.pi_batch_create(boxes, [0.1, 0.2, 0.05, 0.3], ns)
    try:
        rng = np.random.default_rng(0)
        v = rng.standard_normal(sum(ns)).astype(np.float32)
        pos = [torch.from_numpy(rng.random(sum(ns), dtype=np.float32)).to(dev) for _ in range(3)]
        B.pi_batch_bin(ctx, *pos, ns)
        tot = torch.zeros(4, dtype=torch.float64, device=dev)
        B.pi_total_f64(ctx, torch.from_numpy(v).to(dev), tot)
        got = tot.cpu().numpy()
        p = 0
        for k, n in enumerate(ns):
            ref = v[p:p + n].astype(np.float64).sum()
            assert got[k] == pytest.approx(ref, rel=1e-12, abs=1e-12)
            p += n
    finally:
        B.pi_destroy(ctx)

"""Stream order around the dependent launches.

Every kernel of a step after the first may begin while the kernel before it
drains, and the histogram kernel loads its positions before it waits.  These
tests check the orderings that rely on: positions written by another kernel
just before binning, on the same stream, are the ones binned; consecutive
steps on changing positions each see their own binning; back-to-back
interaction calls into different outputs all see the same binning.
"""
import numpy as np

import pytest

from paper_2406_16091_gb300 import binding as B
from paper_2406_16091_gb300 import workloads as W

from gpu_harness import check_interaction, oracle_run, torch_mod

pytestmark = pytest.mark.gpu


def _outputs(torch, dev, n, steps):
    return [[torch.full((n,), float("nan"), device=dev) for _ in range(4)] +
            [torch.full((n,), -1, dtype=torch.int32, device=dev)] for _ in range(steps)]


def _as_dict(o):
    res = {k: v.cpu().numpy() for k, v in zip(("S", "Vx", "Vy", "Vz"), o[:4])}
    res["nbr"] = o[4].cpu().numpy().view(np.uint32)
    return res


@pytest.mark.parametrize("tile", [5, 6])
def test_positions_written_just_before_binning_are_the_ones_binned(tile):
    torch = torch_mod()
    dev = torch.device("cuda", 0)
    w = W.scaled(W.SCALE, 200000)
    n = w.n
    sets = [w.positions(), W.uniform(n, 4242)]
    refs = [oracle_run(*p, w.lo, w.hi, w.rc, w.h) for p in sets]
    src = [[torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(dev) for a in p] for p in sets]
    tx, ty, tz = (torch.empty(n, device=dev) for _ in range(3))
    steps = 6
    outs = _outputs(torch, dev, n, steps)
    ctx = B.pi_create(w.lo, w.hi, w.rc, n)
    try:
        B.pi_set_option(ctx, B.PI_OPT_TILE, tile)
        s = torch.cuda.current_stream()
        torch.cuda.synchronize()
        for k in range(steps):
            # torch elementwise kernels (not copies) on the same stream,
            # directly before k_zero; x * 1 is x exactly
            for d, a in zip((tx, ty, tz), src[k % 2]):
                torch.mul(a, 1.0, out=d)
            B.pi_bin(ctx, tx, ty, tz, n, s)
            B.pi_interact(ctx, w.h, *outs[k], B.PI_ORDER_SORTED, s)
        st, _ = B.pi_sync_status(ctx, s, raise_on_error=False)
        assert st == B.PI_OK, B.status_str(st)
        for k in range(steps):
            check_interaction(_as_dict(outs[k]), refs[k % 2][1])
    finally:
        B.pi_destroy(ctx)


def test_back_to_back_interactions_see_the_same_binning():
    torch = torch_mod()
    dev = torch.device("cuda", 0)
    w = W.scaled(W.SCALE, 100000)
    n = w.n
    x, y, z = w.positions()
    b, r = oracle_run(x, y, z, w.lo, w.hi, w.rc, w.h)
    tx, ty, tz = (torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(dev) for a in (x, y, z))
    calls = 8
    outs = _outputs(torch, dev, n, calls)
    ctx = B.pi_create(w.lo, w.hi, w.rc, n)
    try:
        s = torch.cuda.current_stream()
        B.pi_bin(ctx, tx, ty, tz, n, s)
        # alternate the two direct shapes: each call follows another
        # interaction kernel, not the binning
        for k in range(calls):
            B.pi_set_option(ctx, B.PI_OPT_TILE, 5 + (k & 1))
            B.pi_interact(ctx, w.h, *outs[k], B.PI_ORDER_SORTED, s)
        st, _ = B.pi_sync_status(ctx, s, raise_on_error=False)
        assert st == B.PI_OK, B.status_str(st)
        first = _as_dict(outs[0])
        check_interaction(first, r)
        for k in range(1, calls):
            g = _as_dict(outs[k])
            for name in ("S", "Vx", "Vy", "Vz", "nbr"):
                assert np.array_equal(g[name].view(np.uint32), first[name].view(np.uint32)), (k, name)
    finally:
        B.pi_destroy(ctx)

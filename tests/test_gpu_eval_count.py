"""The evaluation counter of the direct kernels (PI_OPT_COUNT_EVALS,
pi_eval_count): counting leaves every output bit for bit as it was, counts
at least every within-cutoff pair (each is an evaluation of its target),
restarts at every bin and adds up over repeated interactions, and the
shapes that do not count report zero."""
import numpy as np
import pytest

from paper_2406_16091_gb300 import binding as B
from paper_2406_16091_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _run(ctx, torch, t, n, h, s):
    dev = t[0].device
    out = [torch.empty(n, device=dev) for _ in range(4)]
    nb = torch.empty(n, dtype=torch.int32, device=dev)
    B.pi_interact(ctx, h, *out, nb, B.PI_ORDER_SORTED, s)
    B.pi_sync_status(ctx, s)
    return [o.cpu().numpy().view(np.uint32) for o in out] + [nb.cpu().numpy().view(np.uint32)]


@pytest.mark.parametrize("tile", [5, 6])
@pytest.mark.parametrize("name", ["small", "clustered_300000"])
def test_counting_is_exact_and_changes_nothing(tile, name):
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    w = W.SMALL if name == "small" else W.scaled(W.CLUSTERED, 300000)
    x, y, z = w.positions()
    s = torch.cuda.current_stream()
    ctx = B.pi_create(w.lo, w.hi, w.rc, w.n)
    try:
        B.pi_set_option(ctx, B.PI_OPT_TILE, tile)
        t = [torch.from_numpy(a).to(dev) for a in (x, y, z)]
        B.pi_bin(ctx, *t, w.n, s)
        plain = _run(ctx, torch, t, w.n, w.h, s)
        assert B.pi_eval_count(ctx, s) == 0
        B.pi_set_option(ctx, B.PI_OPT_COUNT_EVALS, 1)
        B.pi_bin(ctx, *t, w.n, s)
        counted = _run(ctx, torch, t, w.n, w.h, s)
        for a, b in zip(plain, counted):
            assert np.array_equal(a, b)
        e1 = B.pi_eval_count(ctx, s)
        pairs = int(counted[4].astype(np.int64).sum())
        assert pairs > 0 and pairs <= e1 <= 12 * pairs
        _run(ctx, torch, t, w.n, w.h, s)
        assert B.pi_eval_count(ctx, s) == 2 * e1
        B.pi_bin(ctx, *t, w.n, s)
        assert B.pi_eval_count(ctx, s) == 0
        _run(ctx, torch, t, w.n, w.h, s)
        assert B.pi_eval_count(ctx, s) == e1
        # a staged shape counts nothing
        B.pi_set_option(ctx, B.PI_OPT_TILE, 2)
        B.pi_bin(ctx, *t, w.n, s)
        _run(ctx, torch, t, w.n, w.h, s)
        assert B.pi_eval_count(ctx, s) == 0
        with pytest.raises(B.PiError):
            B.pi_set_option(ctx, B.PI_OPT_COUNT_EVALS, 2)
    finally:
        B.pi_destroy(ctx)


def test_calls_on_a_destroyed_context_raise_on_the_host():
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    w = W.SMALL
    ctx = B.pi_create(w.lo, w.hi, w.rc, w.n)
    B.pi_destroy(ctx)
    t = [torch.zeros(w.n, device=dev) for _ in range(3)]
    with pytest.raises(Exception, match="destroyed"):
        B.pi_bin(ctx, *t, w.n, torch.cuda.current_stream())
    with pytest.raises(Exception, match="destroyed"):
        B.pi_destroy(ctx)

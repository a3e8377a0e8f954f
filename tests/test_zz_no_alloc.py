"""The allocation-free scan entry point, checked against pi_bin's own scan.

pi_scan_counts_noalloc serves callers that cannot allocate device memory;
its scratch is a fixed array inside the library.  This file sorts last so a
run that stops at the first failure has run every other test before it.
"""
import numpy as np
import pytest

from paper_2406_16091_gb300 import binding as B
from paper_2406_16091_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _bin_counts(torch, w):
    """Counts, offsets and M_C from the existing entry point, pi_bin."""
    dev = torch.device("cuda", 0)
    x, y, z = w.positions()
    s = torch.cuda.current_stream()
    ctx = B.pi_create(w.lo, w.hi, w.rc, w.n)
    try:
        tx, ty, tz = (torch.from_numpy(a).to(dev) for a in (x, y, z))
        B.pi_bin(ctx, tx, ty, tz, w.n, s)
        dims = B.pi_grid(ctx)
        C = dims[0] * dims[1] * dims[2]
        counts = torch.empty(C, dtype=torch.int32, device=dev)
        offsets = torch.empty(C + 1, dtype=torch.int32, device=dev)
        B.pi_copy_binned(ctx, counts, offsets, None, None, None, None, s)
        _, mpc = B.pi_sync_status(ctx, s)
    finally:
        B.pi_destroy(ctx)
    return counts, offsets, mpc


def test_noalloc_scan_matches_pi_bin_twice():
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    s = torch.cuda.current_stream()
    # two calls in a row, the second on a different (larger) grid, so the
    # shared scratch is reused with other contents left behind
    for w in (W.scaled(W.CLUSTERED, 300000), W.SCALE):
        counts, ref_offsets, ref_max = _bin_counts(torch, w)
        C = counts.numel()
        offsets = torch.full((C + 1,), -1, dtype=torch.int32, device=dev)
        result = torch.full((2,), -1, dtype=torch.int32, device=dev)
        B.pi_scan_counts_noalloc(counts, C, offsets, result, s)
        torch.cuda.synchronize()
        assert np.array_equal(offsets.cpu().numpy(), ref_offsets.cpu().numpy())
        res = result.cpu().numpy().view(np.uint32)
        assert res[0] == ref_max and res[1] == 0


def test_noalloc_scan_rejects_oversized_grid():
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    buf = torch.zeros(4, dtype=torch.int32, device=dev)
    with pytest.raises(B.PiError) as e:
        B.pi_scan_counts_noalloc(buf, (1 << 24) + 1, buf, None, torch.cuda.current_stream())
    assert e.value.status == B.PI_ERR_CAPACITY
    assert "exceed the fixed scratch limit" in B.last_error()

"""The allocation-free scan entry point, pi_scan_counts_noalloc.

Some callers cannot call cudaMalloc: code whose device memory is reserved up
front by another allocator (a framework's caching allocator, a solver with a
fixed budget), or a latency-critical loop where an allocation could
synchronise the device.  For them the library keeps the scan's scratch in one
fixed array of its own.  These tests compare that entry point with the
oracle's sequential scan (and with pi_bin's own scan) on two calls in a row,
around the 4096-count tile boundaries of the kernel, up to the 2^24-cell
limit, and check the host-side rejections.  The file sorts last, so a run
that stops at the first failure has run every other test before it.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2406_16091_gb300 import binding as B
from paper_2406_16091_gb300 import workloads as W

pytestmark = pytest.mark.gpu

LIMIT = 1 << 24


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


def _scan(torch, counts_np, with_result=True):
    """One call of the entry point on host counts; returns (offsets, result)."""
    dev = torch.device("cuda", 0)
    s = torch.cuda.current_stream()
    C = len(counts_np)
    counts = torch.from_numpy(counts_np.view(np.int32)).to(dev)
    offsets = torch.full((C + 1,), -1, dtype=torch.int32, device=dev)
    result = torch.full((2,), -1, dtype=torch.int32, device=dev) if with_result else None
    B.pi_scan_counts_noalloc(counts, C, offsets, result, s)
    torch.cuda.synchronize()
    res = result.cpu().numpy().view(np.uint32) if with_result else None
    return offsets.cpu().numpy().view(np.uint32), res


def test_noalloc_scan_matches_pi_bin_and_oracle_twice():
    torch = pytest.importorskip("torch")
    # two calls in a row, the second on a different (larger) grid, so the
    # shared scratch is reused with other contents left behind
    for w in (W.scaled(W.CLUSTERED, 300000), W.SCALE):
        counts, ref_offsets, ref_max = _bin_counts(torch, w)
        cnp = counts.cpu().numpy().view(np.uint32).copy()
        got, res = _scan(torch, cnp)
        assert np.array_equal(got, oracle.exclusive_scan(cnp))
        assert np.array_equal(got, ref_offsets.cpu().numpy().view(np.uint32))
        assert res[0] == ref_max == int(cnp.max()) and res[1] == 0


@pytest.mark.parametrize("C", [1, 3, 4095, 4096, 4097, 8191, 8192, 8193, 12288 + 5, LIMIT])
def test_noalloc_scan_tile_edges_against_oracle(C):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(9000 + C % 997)
    for call in range(2):  # two calls in a row on the same shared scratch
        counts = rng.integers(0, 17 if call == 0 else 40, size=C, dtype=np.uint32)
        if C > 2:
            counts[rng.integers(0, C)] = 1000 + call  # a distinct maximum somewhere inside
        got, res = _scan(torch, counts)
        ref = oracle.exclusive_scan(counts)
        assert got[-1] == int(counts.astype(np.int64).sum())
        assert np.array_equal(got, ref), f"C={C}, call {call}"
        assert res[0] == int(counts.max()) and res[1] == 0


def test_noalloc_scan_without_result():
    torch = pytest.importorskip("torch")
    counts = np.random.default_rng(5).integers(0, 9, size=4097, dtype=np.uint32)
    got, _ = _scan(torch, counts, with_result=False)
    assert np.array_equal(got, oracle.exclusive_scan(counts))


def test_noalloc_scan_rejects_misaligned_view():
    """A view that starts one element in is 4-byte but not 16-byte aligned:
    the library refuses it on the host, before anything is enqueued."""
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    s = torch.cuda.current_stream()
    base = torch.arange(1, 4102, dtype=torch.int32, device=dev)
    out = torch.full((4102,), -7, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    for counts, offsets in ((base[1:], out[:4101]), (base[:4100], out[1:])):
        with pytest.raises(B.PiError) as e:
            B.pi_scan_counts_noalloc(counts, 4100, offsets, None, s)
        assert e.value.status == B.PI_ERR_INVALID_ARG
        assert "16-byte aligned" in B.last_error()
    torch.cuda.synchronize()
    assert bool((out == -7).all()), "a rejected call wrote the offsets"


def test_noalloc_scan_rejects_oversized_grid():
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    buf = torch.zeros(4, dtype=torch.int32, device=dev)
    # through the C ABI itself: the library refuses the size before touching
    # the (too short) buffers
    st = B.load().pi_scan_counts_noalloc(ctypes.c_void_p(buf.data_ptr()), LIMIT + 1,
                                         ctypes.c_void_p(buf.data_ptr()), None, None)
    assert st == B.PI_ERR_CAPACITY
    assert "exceed the fixed scratch limit" in B.last_error()
    # the binding refuses buffers shorter than C before calling the library
    with pytest.raises(ValueError):
        B.pi_scan_counts_noalloc(buf, 5, buf, None, torch.cuda.current_stream())

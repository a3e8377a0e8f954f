"""Serving: jobs of different size, box, cutoff and layout arrive over time;
each result is the same as the job run alone, and the statistics are
reported."""
import numpy as np
import pytest

import oracle
from paper_2406_16091_gb300 import binding as B
from paper_2406_16091_gb300 import workloads as W

from gpu_harness import check_interaction

pytestmark = pytest.mark.gpu


def _jobs(count=36, seed=9):
    from paper_2406_16091_gb300.serving import make_job

    rng = np.random.default_rng(seed)
    jobs = []
    for k in range(count):
        n = int(np.exp(rng.uniform(np.log(200), np.log(60000))))
        if k == 5:
            n = 0
        cells = int(rng.integers(3, 30))
        sysk = W._system_for(max(n, 1), max(n, 1) / cells ** 3, 7000 + k,
                             "clustered" if k % 3 == 0 else "uniform")
        x, y, z = W.uniform(n, 7000 + k) if sysk.layout == "uniform" else W.clustered(max(n, 1), 7000 + k)
        x, y, z = x[:n], y[:n], z[:n]
        jobs.append(make_job(k, x, y, z, (0, 0, 0), (1, 1, 1), sysk.rc, sysk.h,
                             arrival=float(k) * 0.002))
    return jobs


def _alone(job):
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    n = job.n
    ctx = B.pi_create(job.lo, job.hi, job.rc, max(n, 1))
    try:
        t = [job.x.to(dev), job.y.to(dev), job.z.to(dev)]
        out = [torch.empty(max(n, 1), device=dev) for _ in range(4)]
        nb = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
        B.pi_bin(ctx, *t, n)
        if n:
            B.pi_interact(ctx, job.h, *out, nb, B.PI_ORDER_ORIGINAL)
        B.pi_sync_status(ctx)
        return [o.cpu()[:n].numpy() for o in out] + [nb.cpu()[:n].numpy()]
    finally:
        B.pi_destroy(ctx)


def test_results_in_the_mix_equal_results_alone():
    pytest.importorskip("torch")
    from paper_2406_16091_gb300.serving import Server

    jobs = _jobs()
    srv = Server(buckets=((16384, 1), (65536, 2)), max_slots_per_bucket=3)
    try:
        stats = srv.run(jobs)
    finally:
        srv.close()
    assert stats["jobs"] == len(jobs)
    assert 0 < stats["p50_ms"] <= stats["p99_ms"]
    for job in jobs:
        assert job.t_done >= job.t_start >= job.arrival
        n = job.n
        mix = [job.S[:n].numpy(), job.Vx[:n].numpy(), job.Vy[:n].numpy(), job.Vz[:n].numpy(),
               job.nbr[:n].numpy()]
        alone = _alone(job)
        for a, b in zip(mix, alone):
            assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    # and a few of them against the oracle
    for job in jobs[1:6]:
        n = job.n
        x, y, z = job.x[:n].numpy(), job.y[:n].numpy(), job.z[:n].numpy()
        b = oracle.bin_particles(x, y, z, job.lo, job.hi, job.rc)
        r = oracle.interact(b, job.rc, job.h)
        g = {"S": job.S[:n].numpy(), "Vx": job.Vx[:n].numpy(), "Vy": job.Vy[:n].numpy(),
             "Vz": job.Vz[:n].numpy(), "nbr": job.nbr[:n].numpy().view(np.uint32)}
        check_interaction(g, r, perm=b.perm)


def test_memory_budget_limits_slots_and_jobs_wait():
    pytest.importorskip("torch")
    from paper_2406_16091_gb300.serving import Server, slot_bytes

    jobs = _jobs(count=10, seed=3)
    for j in jobs:
        j.arrival = 0.0
    budget = slot_bytes(65536, 65536) + 1
    srv = Server(buckets=((65536, 1),), hbm_budget=budget, max_slots_per_bucket=8)
    try:
        stats = srv.run(jobs)
    finally:
        srv.close()
    assert stats["slots"] == {65536: 1}
    assert stats["jobs"] == 10


def test_submit_host_checks_the_grid_capacity():
    torch = pytest.importorskip("torch")
    ctx = B.pi_create((0, 0, 0), (1, 1, 1), W.rc_for_cells(8), 1000)
    try:
        x = torch.zeros(10).pin_memory()
        out = [torch.empty(10).pin_memory() for _ in range(4)]
        nb = torch.empty(10, dtype=torch.int32).pin_memory()
        # 16^3 cells do not fit a context sized for 8^3
        with pytest.raises(B.PiError) as e:
            B.pi_submit_host(ctx, (0, 0, 0), (1, 1, 1), W.rc_for_cells(16), x, x, x, 10, 0.03, *out, nb)
        assert e.value.status == B.PI_ERR_CAPACITY
        # 4^3 cells do: the job runs and matches the oracle's counts
        xs = W.uniform(10, 42)
        t = [torch.from_numpy(a).pin_memory() for a in xs]
        rc = W.rc_for_cells(4)
        B.pi_submit_host(ctx, (0, 0, 0), (1, 1, 1), rc, *t, 10, rc / 2, *out, nb)
        B.pi_sync_status(ctx)
        b = oracle.bin_particles(*xs, (0, 0, 0), (1, 1, 1), rc)
        r = oracle.interact(b, rc, rc / 2)
        assert np.array_equal(nb.numpy().view(np.uint32)[b.perm], r.nbr)
    finally:
        B.pi_destroy(ctx)


@pytest.mark.parametrize("n", [0, 1, 3, 1000, 4099])
def test_strided_host_step_equals_separate_arrays(n):
    """One block each way (one copy in, one out) gives bit for bit the
    results of separate arrays; bad strides and arrays off their stride are
    rejected before anything is enqueued."""
    torch = pytest.importorskip("torch")
    w = W.scaled(W.SMALL, max(n, 1))
    x, y, z = (a[:n] for a in w.positions())
    cap = 4100
    ctx = B.pi_create(w.lo, w.hi, w.rc, cap)
    try:
        d = max(4, (n + 3) // 4 * 4)
        blk = torch.zeros(3 * d).pin_memory()
        for k, a in enumerate((x, y, z)):
            blk[k * d:k * d + n] = torch.from_numpy(a)
        outb = torch.full((5 * d,), float("nan")).pin_memory()
        # addresses inside the blocks (slices of no elements may not carry one)
        ib, ob = blk.data_ptr(), outb.data_ptr()

        def at(base, s, k):
            return base + 4 * s * k

        B.pi_submit_host_strided(ctx, w.lo, w.hi, w.rc, at(ib, d, 0), at(ib, d, 1), at(ib, d, 2), d, n, w.h,
                                 *(at(ob, d, k) for k in range(5)), d)
        B.pi_sync_status(ctx)
        o = [outb[k * d:k * d + n] for k in range(4)] + [outb[4 * d:4 * d + n].view(torch.int32)]
        sep = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (x, y, z)]
        ref = [torch.empty(max(n, 1)).pin_memory() for _ in range(4)]
        rnb = torch.empty(max(n, 1), dtype=torch.int32).pin_memory()
        B.pi_run_host(ctx, *sep, n, w.h, *ref, rnb)
        for a, b in zip(o, ref + [rnb]):
            assert np.array_equal(a.numpy().view(np.uint32), b[:n].numpy().view(np.uint32))
        bad = [(d + 2, d + 2),                       # not a multiple of 4
               (d, (cap + 4 + 3) // 4 * 4 + 4)]      # beyond the staging arrays
        if n > 4:
            bad.append((n - 1 - (n - 1) % 4, d))     # below n
        for si, so in bad:
            with pytest.raises(B.PiError) as e:
                B.pi_submit_host_strided(ctx, w.lo, w.hi, w.rc, at(ib, si, 0), at(ib, si, 1), at(ib, si, 2), si,
                                         n, w.h, *(at(ob, so, k) for k in range(5)), so)
            assert e.value.status == B.PI_ERR_INVALID_ARG
        # y not at x + stride
        with pytest.raises(B.PiError) as e:
            B.pi_submit_host_strided(ctx, w.lo, w.hi, w.rc, at(ib, d, 0), at(ib, d, 2), at(ib, d, 2), d, n, w.h,
                                     *(at(ob, d, k) for k in range(5)), d)
        assert e.value.status == B.PI_ERR_INVALID_ARG
    finally:
        B.pi_destroy(ctx)

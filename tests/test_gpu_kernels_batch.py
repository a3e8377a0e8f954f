"""GPU parity for the other interaction kernels (Sec. 7.1-7.2) and for
batches of independent systems run in one launch per kernel."""
import numpy as np
import pytest

import oracle
from paper_2406_16091_gb300 import binding as B
from paper_2406_16091_gb300 import workloads as W

from gpu_harness import TOL, check_binning, check_interaction, oracle_run, run_gpu

pytestmark = pytest.mark.gpu

KERNELS = [(B.PI_KERNEL_LJ, oracle.LJ), (B.PI_KERNEL_LOWFLOP, oracle.LOWFLOP),
           (B.PI_KERNEL_HIGHFLOP, oracle.HIGHFLOP), (B.PI_KERNEL_GAUSSIAN, oracle.GAUSSIAN)]


# (algorithm, tile shape): the staged one-target shape, the direct kernel
# (two targets per thread, packed), Alg. 1
PATHS = [(B.PI_ALGO_TILED, 2), (B.PI_ALGO_TILED, 5), (B.PI_ALGO_TILED, 6), (B.PI_ALGO_PPNL, None)]


@pytest.mark.parametrize("path", PATHS, ids=["staged", "direct", "direct4", "ppnl"])
@pytest.mark.parametrize("kern", KERNELS)
@pytest.mark.parametrize("precision", [B.PI_PREC_FP32, B.PI_PREC_KAHAN])
def test_kernel_parity(path, kern, precision):
    gk, ok = kern
    algo, tile = path
    w = W.scaled(W.SMALL, 20000)
    x, y, z = w.positions()
    b, r = oracle_run(x, y, z, w.lo, w.hi, w.rc, w.h, ok)
    g = run_gpu(x, y, z, w.lo, w.hi, w.rc, w.h, algo=algo, precision=precision, kernel=gk, tile=tile)
    check_binning(g, b)
    check_interaction(g, r)


def _dense_cluster():
    """Background plus one tight cluster: cells of several hundred members,
    so the direct kernel takes exact window bounds in them."""
    rng = np.random.default_rng(3)
    bg = rng.random((20000, 3)).astype(np.float32)
    cl = (0.5 + 0.004 * rng.standard_normal((6000, 3))).astype(np.float32)
    p = np.concatenate([bg, cl])
    return p[:, 0].copy(), p[:, 1].copy(), p[:, 2].copy(), (0, 0, 0), (1, 1, 1), 1.0 / 64


@pytest.mark.parametrize("kern", KERNELS)
@pytest.mark.parametrize("precision", [B.PI_PREC_FP32, B.PI_PREC_KAHAN])
def test_dense_cells_exact_windows_bitwise_equal(kern, precision):
    """Cells above 255 members: the direct kernel's binary-searched window
    bounds (tighter than whole cells) give the staged path's sums bit for
    bit, and both match the oracle."""
    gk, ok = kern
    x, y, z, lo, hi, rc = _dense_cluster()
    b, r = oracle_run(x, y, z, lo, hi, rc, rc / 2, ok)
    assert b.max_per_cell > 255
    res = {t: run_gpu(x, y, z, lo, hi, rc, rc / 2, precision=precision, kernel=gk, tile=t, binned=False)
           for t in (2, 5, 6)}
    for t in (5, 6):
        for k in ("S", "Vx", "Vy", "Vz", "nbr"):
            assert np.array_equal(res[2][k].view(np.uint32), res[t][k].view(np.uint32)), (t, k)
    # Plain FP32 sums of up to m terms carry the sequential-summation bound
    # (m + 1) 2^-24 of sum|terms| (one rounding per term and per add); with
    # several hundred neighbours of the Lennard-Jones kernel's wide range that
    # bound, not 1e-5, is what FP32 can promise.  The compensated sums keep
    # 1e-5 at any count.
    m = int(r.nbr.max())
    tol = TOL if precision == B.PI_PREC_KAHAN else max(TOL, 1.1 * (m + 2) * 2.0 ** -24)
    check_interaction(res[5], r, tol=tol)


@pytest.mark.parametrize("kern", KERNELS)
@pytest.mark.parametrize("precision", [B.PI_PREC_FP32, B.PI_PREC_KAHAN])
def test_staged_and_direct_paths_bitwise_equal(kern, precision):
    """Every target's terms are summed in the order of its own windows on
    every path; candidates a path reads beyond them (the other target's of a
    packed pair, sentinel slots, the target itself) are exact no-ops, also
    for the compensated sums.  So the one-target staged path and the packed
    two-target direct kernel agree bit for bit, for every kernel and both
    precision modes, on a clustered layout with dense cells."""
    gk, ok = kern
    w = W.scaled(W.CLUSTERED, 40000)
    x, y, z = w.positions()
    _, r = oracle_run(x, y, z, w.lo, w.hi, w.rc, w.h, ok)
    res = {t: run_gpu(x, y, z, w.lo, w.hi, w.rc, w.h, precision=precision, kernel=gk, tile=t, binned=False)
           for t in (0, 2, 3, 5, 6)}
    for t in (0, 3, 5, 6):
        for k in ("S", "Vx", "Vy", "Vz", "nbr"):
            assert np.array_equal(res[2][k].view(np.uint32), res[t][k].view(np.uint32)), (t, k)
    check_interaction(res[5], r)


def _systems(seed=5):
    """Uneven systems: different sizes, boxes, cutoffs, layouts, an empty one."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(12):
        n = int(np.exp(rng.uniform(np.log(300), np.log(30000))))
        if k == 3:
            n = 0
        if k == 4:
            n = 1
        cells = int(rng.integers(3, 24))
        lo = tuple(float(v) for v in rng.uniform(-2, 2, 3).astype(np.float32))
        ext = float(rng.uniform(0.5, 2.0))
        hi = tuple(float(np.float32(v + ext)) for v in lo)
        rc = W.rc_for_cells(cells, ext) * 0.999
        if k % 4 == 1 and n > 10:
            x, y, z = W.clustered(n, 100 + k)
            x = (np.float32(lo[0]) + np.float32(ext) * x).astype(np.float32)
            y = (np.float32(lo[1]) + np.float32(ext) * y).astype(np.float32)
            z = (np.float32(lo[2]) + np.float32(ext) * z).astype(np.float32)
            x = np.minimum(x, np.nextafter(np.float32(hi[0]), np.float32(lo[0])))
            y = np.minimum(y, np.nextafter(np.float32(hi[1]), np.float32(lo[1])))
            z = np.minimum(z, np.nextafter(np.float32(hi[2]), np.float32(lo[2])))
        else:
            x, y, z = W.uniform(n, 100 + k, lo, hi)
        out.append(dict(n=n, lo=lo, hi=hi, rc=rc, h=rc / 2, x=x, y=y, z=z))
    return out


@pytest.mark.parametrize("algo", [(B.PI_ALGO_TILED, None), (B.PI_ALGO_TILED, 6), (B.PI_ALGO_TILED, 2),
                                  (B.PI_ALGO_PPNL, None)], ids=["direct", "direct4", "staged", "ppnl"])
@pytest.mark.parametrize("order", [B.PI_ORDER_SORTED, B.PI_ORDER_ORIGINAL])
@pytest.mark.parametrize("binning", [B.PI_BIN_PER_PARTICLE, B.PI_BIN_RADIX, B.PI_BIN_BUCKETED],
                         ids=["per_particle", "radix", "bucketed"])
def test_batch_matches_each_system_alone(algo, order, binning):
    algo, tile = algo
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    systems = _systems()
    ns = [s["n"] for s in systems]
    N = sum(ns)
    ctx = B.pi_batch_create([(s["lo"], s["hi"]) for s in systems], [s["rc"] for s in systems],
                            [n + 5 for n in ns])
    try:
        B.pi_set_option(ctx, B.PI_OPT_ALGO, algo)
        B.pi_set_option(ctx, B.PI_OPT_BINNING, binning)
        if tile is not None:
            B.pi_set_option(ctx, B.PI_OPT_TILE, tile)
        S_, C, _ = B.pi_batch_info(ctx)
        assert S_ == len(systems)
        cat = lambda k: torch.from_numpy(np.concatenate([s[k] for s in systems]).astype(np.float32)).to(dev)
        st = torch.cuda.current_stream()
        tx, ty, tz = cat("x"), cat("y"), cat("z")
        out = [torch.full((N,), float("nan"), device=dev) for _ in range(4)]
        nb = torch.full((N,), -1, dtype=torch.int32, device=dev)
        B.pi_batch_bin(ctx, tx, ty, tz, ns, st)
        B.pi_batch_interact(ctx, [s["h"] for s in systems], *out, nb, order, st)
        counts = torch.empty(C, dtype=torch.int32, device=dev)
        offsets = torch.empty(C + 1, dtype=torch.int32, device=dev)
        perm = torch.empty(max(N, 1), dtype=torch.int32, device=dev)
        B.pi_copy_binned(ctx, counts, offsets, perm, None, None, None, st)
        status, mpc = B.pi_sync_status(ctx, st, raise_on_error=False)
        assert status == B.PI_OK
        counts = counts.cpu().numpy().view(np.uint32)
        offsets = offsets.cpu().numpy().view(np.uint32)
        perm = perm.cpu().numpy().view(np.uint32)[:N]
        outs = [o.cpu().numpy() for o in out]
        nbr = nb.cpu().numpy().view(np.uint32)
        p0 = c0 = 0
        best_mpc = 0
        for k, s in enumerate(systems):
            b, r = oracle_run(s["x"], s["y"], s["z"], s["lo"], s["hi"], s["rc"], s["h"])
            dims = B.pi_batch_grid(ctx, k)
            assert tuple(dims) == tuple(b.dims)
            c1 = c0 + int(np.prod(dims))
            n = s["n"]
            assert np.array_equal(counts[c0:c1], b.counts)
            assert np.array_equal(offsets[c0:c1 + 1] - p0, b.offsets)
            assert np.array_equal(perm[p0:p0 + n] - p0, b.perm)
            best_mpc = max(best_mpc, b.max_per_cell)
            if n:
                sl = slice(p0, p0 + n)
                g = {"S": outs[0][sl], "Vx": outs[1][sl], "Vy": outs[2][sl], "Vz": outs[3][sl],
                     "nbr": nbr[sl]}
                check_interaction(g, r, perm=b.perm if order == B.PI_ORDER_ORIGINAL else None)
            p0 += n
            c0 = c1
        assert c0 == C and mpc == best_mpc
    finally:
        B.pi_destroy(ctx)


def test_batch_rejects_bad_counts():
    torch = pytest.importorskip("torch")
    ctx = B.pi_batch_create([((0, 0, 0), (1, 1, 1))] * 2, [0.1, 0.2], [10, 10])
    try:
        buf = torch.zeros(32, device="cuda")
        with pytest.raises(B.PiError) as e:
            B.pi_batch_bin(ctx, buf, buf, buf, [5, 11])
        assert e.value.status == B.PI_ERR_CAPACITY
        with pytest.raises(B.PiError):
            B.pi_bin(ctx, buf, buf, buf, 3)  # single-system call on a batch
    finally:
        B.pi_destroy(ctx)


def _mixed_occupancy_systems(count=24, seed=1004):
    """A scaled-down copy of the batched workload: N log-uniform in [1024,
    40000], mean occupancy uniform in [2, 16], each in its own unit box."""
    systems = W.batched_systems(count=count, seed=seed, n_hi=40000)
    out = []
    for sy in systems:
        x, y, z = sy.positions()
        out.append(dict(n=sy.n, lo=sy.lo, hi=sy.hi, rc=sy.rc, h=sy.h, x=x, y=y, z=z))
    return out


def _check_batch_outputs(systems, outs, nbr):
    p0 = 0
    for s in systems:
        b, r = oracle_run(s["x"], s["y"], s["z"], s["lo"], s["hi"], s["rc"], s["h"])
        n = s["n"]
        sl = slice(p0, p0 + n)
        g = {"S": outs[0][sl], "Vx": outs[1][sl], "Vy": outs[2][sl], "Vz": outs[3][sl], "nbr": nbr[sl]}
        check_interaction(g, r)
        p0 += n


def test_batch_graph_replay_matches_oracle():
    """pi_batch_bin + pi_batch_interact captured in one CUDA graph after
    pi_autotune (which may keep a shape per occupancy regime), replayed twice;
    every system of both replays against the oracle."""
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    systems = _mixed_occupancy_systems()
    ns = [s["n"] for s in systems]
    N = sum(ns)
    hs = [s["h"] for s in systems]
    ctx = B.pi_batch_create([(s["lo"], s["hi"]) for s in systems], [s["rc"] for s in systems], ns)
    try:
        cat = lambda k: torch.from_numpy(np.concatenate([s[k] for s in systems]).astype(np.float32)).to(dev)
        tx, ty, tz = cat("x"), cat("y"), cat("z")
        out = [torch.empty(N, device=dev) for _ in range(4)]
        nb = torch.empty(N, dtype=torch.int32, device=dev)
        cs = torch.cuda.Stream()
        cs.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(cs):
            B.pi_batch_bin(ctx, tx, ty, tz, ns, cs)
            chosen, ms = B.pi_autotune(ctx, hs, *out, nb, B.PI_ORDER_SORTED, 2, cs)
            assert len(ms) == B.PI_NUM_TILES + 2 and ms[B.PI_AUTOTUNE_REGIMES] > 0
            tiles = B.pi_batch_tiles(ctx, len(systems))
            if chosen == B.PI_AUTOTUNE_REGIMES:
                assert set(tiles) <= {5, 6}
            else:
                assert tiles == [-1] * len(systems)
            # an eager step first (writes the range lists the graph replays)
            B.pi_batch_bin(ctx, tx, ty, tz, ns, cs)
            B.pi_batch_interact(ctx, hs, *out, nb, B.PI_ORDER_SORTED, cs)
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=cs):
                B.pi_batch_bin(ctx, tx, ty, tz, ns, cs)
                B.pi_batch_interact(ctx, hs, *out, nb, B.PI_ORDER_SORTED, cs)
        for _ in range(2):
            for o in out:
                o.fill_(float("nan"))
            nb.fill_(-1)
            g.replay()
            torch.cuda.synchronize()
            status, _ = B.pi_sync_status(ctx, torch.cuda.current_stream(), raise_on_error=False)
            assert status == B.PI_OK
            _check_batch_outputs(systems, [o.cpu().numpy() for o in out], nb.cpu().numpy().view(np.uint32))
        del g
    finally:
        B.pi_destroy(ctx)


@pytest.mark.parametrize("kern,prec,order,hdiv", [
    ((B.PI_KERNEL_GAUSSIAN, oracle.GAUSSIAN), B.PI_PREC_FP32, B.PI_ORDER_SORTED, 2),
    ((B.PI_KERNEL_GAUSSIAN, oracle.GAUSSIAN), B.PI_PREC_KAHAN, B.PI_ORDER_ORIGINAL, 2),
    ((B.PI_KERNEL_GAUSSIAN, oracle.GAUSSIAN), B.PI_PREC_FP32, B.PI_ORDER_SORTED, 8),   # compensated exponent
    ((B.PI_KERNEL_LJ, oracle.LJ), B.PI_PREC_FP32, B.PI_ORDER_ORIGINAL, 2),
], ids=["gauss", "kahan-original", "short-h", "lj-original"])
def test_batch_per_system_shapes_bitwise_equal(kern, prec, order, hdiv):
    """A plan that mixes the two- and four-target shapes over the systems
    gives the same outputs bit for bit as one shape for all, and the oracle's
    values; clearing the plan restores the context's shape."""
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    systems = _mixed_occupancy_systems(count=16, seed=77)
    systems[5]["n"] = 0  # a system without particles inside a plan
    for k in "xyz":
        systems[5][k] = systems[5][k][:0]
    for sy in systems:
        sy["h"] = sy["rc"] / hdiv
    ns = [s["n"] for s in systems]
    N = sum(ns)
    hs = [s["h"] for s in systems]
    gk, ok = kern
    ctx = B.pi_batch_create([(s["lo"], s["hi"]) for s in systems], [s["rc"] for s in systems],
                            [max(n, 1) for n in ns])
    try:
        B.pi_set_option(ctx, B.PI_OPT_KERNEL, gk)
        B.pi_set_option(ctx, B.PI_OPT_PRECISION, prec)
        st = torch.cuda.current_stream()
        cat = lambda k: torch.from_numpy(np.concatenate([s[k] for s in systems]).astype(np.float32)).to(dev)
        tx, ty, tz = cat("x"), cat("y"), cat("z")
        B.pi_batch_bin(ctx, tx, ty, tz, ns, st)

        def run():
            out = [torch.full((N,), float("nan"), device=dev) for _ in range(4)]
            nb = torch.full((N,), -1, dtype=torch.int32, device=dev)
            B.pi_batch_interact(ctx, hs, *out, nb, order, st)
            B.pi_sync_status(ctx, st)
            return [o.cpu().numpy().view(np.uint32) for o in out] + [nb.cpu().numpy().view(np.uint32)]

        B.pi_set_option(ctx, B.PI_OPT_TILE, 5)
        ref = run()
        for plan in ([5, 6] * 8, [6] * 16, [6, 6, 5, 5, 5, 6, 6, 6, 5, 6, 5, 5, 6, 5, 6, 6]):
            B.pi_batch_set_tiles(ctx, plan)
            assert B.pi_batch_tiles(ctx, 16) == plan
            got = run()
            for a, b in zip(got, ref):
                assert np.array_equal(a, b)
        # against the oracle, system by system
        outs = [a.view(np.float32) for a in got[:4]]
        p0 = 0
        for sy in systems:
            n = sy["n"]
            if n:
                b, r = oracle_run(sy["x"], sy["y"], sy["z"], sy["lo"], sy["hi"], sy["rc"], sy["h"], ok)
                sl = slice(p0, p0 + n)
                g = {"S": outs[0][sl], "Vx": outs[1][sl], "Vy": outs[2][sl], "Vz": outs[3][sl], "nbr": got[4][sl]}
                if order == B.PI_ORDER_ORIGINAL:
                    check_interaction(g, r, perm=b.perm, rc=sy["rc"])
                else:
                    check_interaction(g, r, rc=sy["rc"])
            p0 += n
        B.pi_batch_set_tiles(ctx, None)
        assert B.pi_batch_tiles(ctx, 16) == [-1] * 16
        with pytest.raises(B.PiError):
            B.pi_batch_set_tiles(ctx, [5] * 15 + [2])
    finally:
        B.pi_destroy(ctx)

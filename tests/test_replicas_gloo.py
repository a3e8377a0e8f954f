"""The multi-GPU form (independent replicas, weak scaling) on CPU process
groups: two gloo ranks run the host logic bench.py uses over NCCL -- the
slowest rank's time, the sum of all ranks' units, the whole-job rate -- and
get replica systems of the same shape but different particles."""
import json
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2406_16091_gb300 import replicas  # noqa: E402
from paper_2406_16091_gb300 import workloads as W  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, outdir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r takes (r + 1) seconds and processes 10 ** r units per step
        t, u = replicas.aggregate(float(rank + 1), float(10 ** rank), torch.device("cpu"))
        w = W.scaled(W.SMALL, 4096)
        x, y, z = replicas.replica_positions(w, rank)
        gathered = [None] * world
        dist.all_gather_object(gathered, (float(x[:8].sum()), len(x)))
        with open(os.path.join(outdir, f"rank{rank}.json"), "w") as f:
            json.dump([t, u, replicas.job_rate(u, 5, t), gathered], f)
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation_and_replicas(tmp_path):
    world = 2
    port = _free_port()
    mp.spawn(_worker, args=(world, port, str(tmp_path)), nprocs=world, join=True)
    for rank in range(world):
        t, u, rate, gathered = json.load(open(tmp_path / f"rank{rank}.json"))
        assert t == 2.0            # the slowest rank's time
        assert u == 11.0           # 1 + 10 units per step
        assert rate == pytest.approx(11.0 * 5 / 2.0)
        (s0, n0), (s1, n1) = gathered
        assert n0 == n1 == 4096    # same shape on every rank
        assert s0 != s1            # independent particles


def test_single_process_is_identity():
    assert replicas.aggregate(3.5, 7) == (3.5, 7.0)
    assert replicas.job_rate(7.0, 2, 3.5) == 4.0
    with pytest.raises(ValueError):
        replicas.job_rate(1.0, 1, 0.0)


def test_rank0_replica_is_the_workload():
    w = W.scaled(W.CLUSTERED, 5000)
    a = replicas.replica_positions(w, 0)
    b = w.positions()
    for p, q in zip(a, b):
        assert np.array_equal(p, q)
    c = replicas.replica_positions(w, 3)
    assert not np.array_equal(a[0], c[0])
    assert all(len(v) == w.n for v in c)
    assert all(float(v.min()) >= 0.0 and float(v.max()) < 1.0 for v in c)

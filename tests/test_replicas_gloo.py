"""The replica (N > 1) host logic on the CPU: two gloo ranks, as bench.py
runs N processes (one per GPU) under torchrun -- max-over-ranks timing, the
whole-job rate, round-robin sharding of independent instances."""
from __future__ import annotations

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1411_7018_gb300 import replicas


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, lr, w = replicas.rank_info()
        # each rank "measures" its own time; the job's time is the slowest rank's
        t = replicas.max_over_ranks(10.0 + 5.0 * r)
        replicas.barrier()
        mine = replicas.shard(range(64), r, w)
        n_all = torch.tensor([len(mine)], dtype=torch.int64)
        dist.all_reduce(n_all)
        out.put((r, lr, w, t, replicas.whole_job_rate(1000.0, t, w), sorted(mine)[:3], int(n_all.item())))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [x[0] for x in res] == [0, 1] and all(x[2] == 2 for x in res)
    assert all(x[3] == 15.0 for x in res)                    # max over ranks
    assert all(abs(x[4] - 2 * 1000.0 / 15.0) < 1e-12 for x in res)
    assert res[0][5] == [0, 2, 4] and res[1][5] == [1, 3, 5]
    assert all(x[6] == 64 for x in res)                       # every instance exactly once


def test_single_process_defaults():
    assert replicas.rank_info({}) == (0, 0, 1)
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.whole_job_rate(100.0, 2.0, 4) == 200.0

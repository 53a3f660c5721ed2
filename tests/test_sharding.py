"""Sharding of independent problems over ranks: partition balance and the
world_size-2 reduction of timing and work over gloo on CPU."""
import os
import socket

import pytest

from paper_1908_03876_gb300 import sharding
from paper_1908_03876_gb300 import workloads as W


def test_partition_covers_and_balances():
    ws = W.batch_workloads(64, N=10, seed=3)
    costs = [sharding.problem_cost(w) for w in ws]
    for world in (1, 2, 3, 8):
        parts = sharding.partition(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(ws)))
        loads = [sum(costs[i] for i in p) for p in parts]
        # LPT bound: no rank above the mean by more than the largest single job
        assert max(loads) <= sum(costs) / world + max(costs)
        assert sharding.partition(costs, world) == parts  # deterministic


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws = W.batch_workloads(16, N=10, seed=3)
    mine = sharding.my_problems(ws, rank, world)
    work = sum(sharding.problem_cost(w) for w in mine)
    ms, total = sharding.aggregate(10.0 + rank, work)
    q.put((rank, [w.name for w in mine], ms, total))
    dist.destroy_process_group()


def test_two_rank_gloo_aggregation():
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ws = W.batch_workloads(16, N=10, seed=3)
    total = sum(sharding.problem_cost(w) for w in ws)
    names = out[0][1] + out[1][1]
    assert sorted(names) == sorted(w.name for w in ws) and not set(out[0][1]) & set(out[1][1])
    for rank, _, ms, tot in out:
        assert ms == 11.0 and tot == total

"""Sharding independent control problems over ranks (one GPU per rank).

Problems are independent, so ranks exchange nothing on the data path: each
rank solves its own share and only the timing and the node counts are reduced
(max of the times, sum of the work) for the aggregate throughput.
"""
from __future__ import annotations

import heapq


def problem_cost(w) -> float:
    """Work of one problem: lattice nodes x time steps."""
    return float(w.nx * w.ny * w.N)


def partition(costs, world: int):
    """Longest-processing-time greedy partition: indices per rank, each rank's
    list in ascending index order.  Deterministic (ties by index and rank)."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0.0, r) for r in range(world)]
    heapq.heapify(heap)
    shares = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        shares[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    return [sorted(s) for s in shares]


def my_problems(workloads, rank: int, world: int):
    parts = partition([problem_cost(w) for w in workloads], world)
    return [workloads[i] for i in parts[rank]]


def aggregate(ms: float, work: float, group=None):
    """(max time over ranks, total work over ranks); identity without a process group."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return ms, work
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    n = torch.tensor([work], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(n, group=group)
    return float(t.item()), float(n.item())

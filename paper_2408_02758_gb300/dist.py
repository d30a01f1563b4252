"""Multi-process (one process per GPU) plumbing for the FTLE benchmarks.

The FTLE path shards without any data-path collective: independent problems (a replica of the
workload per rank, or a share of a batch's instances) run on separate GPUs, and the only
communication is host-side control: a barrier around the timed region and the maximum of the
per-rank times.  Ranks are launched by torch.distributed.run (RANK, LOCAL_RANK, WORLD_SIZE,
MASTER_ADDR, MASTER_PORT in the environment); NCCL is used between GPUs, gloo on CPU.
"""
from __future__ import annotations

import heapq
import os
from dataclasses import dataclass


@dataclass
class Ranks:
    world: int
    rank: int
    local: int


def from_env() -> Ranks:
    return Ranks(int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
                 int(os.environ.get("LOCAL_RANK", "0")))


def init(ranks: Ranks, backend: str, device=None):
    """Join the process group (no-op for a single rank); the rendezvous defaults to 127.0.0.1."""
    if ranks.world <= 1:
        return
    import torch.distributed as dist

    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    if dist.is_initialized():
        return
    kw = {"device_id": device} if (backend == "nccl" and device is not None) else {}
    dist.init_process_group(backend, rank=ranks.rank, world_size=ranks.world, **kw)


def barrier(ranks: Ranks):
    if ranks.world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(value: float, ranks: Ranks, device="cpu") -> float:
    """The largest of the ranks' values (e.g. the slowest rank's time per step)."""
    if ranks.world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, ranks: Ranks, device="cpu") -> float:
    if ranks.world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def lpt_assign(costs, world: int) -> list[list[int]]:
    """Longest-processing-time-first assignment of items to `world` bins: items in decreasing
    cost order each go to the currently lightest bin (ties to the lower bin index).  Every rank
    computes the same assignment from the same costs."""
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    heap = [(0.0, r) for r in range(world)]
    bins: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        bins[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    return [sorted(b) for b in bins]

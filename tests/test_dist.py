"""Multi-rank host logic on CPU: two gloo ranks exchange the max of their step times, pass a
barrier, and agree on the LPT assignment of batch instances (no GPU, no data-path collective)."""
import os
import socket

import pytest


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import torch.distributed as dist

    from paper_2408_02758_gb300 import dist as D
    from paper_2408_02758_gb300 import inputs as I

    r = D.from_env()
    D.init(r, "gloo")
    try:
        D.barrier(r)
        slowest = D.max_over_ranks(10.0 + 5.0 * rank, r)
        total = D.sum_over_ranks(100.0 * (rank + 1), r)
        batch = I.batched_preset(16, scale=1 / 8)
        costs = [w.mesh.n_nodes * w.n_steps for w in batch]
        mine = D.lpt_assign(costs, r.world)[r.rank]
        q.put((rank, slowest, total, mine))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert out[0][1] == out[1][1] == 15.0
    assert out[0][2] == out[1][2] == 300.0
    a, b = out[0][3], out[1][3]
    assert not set(a) & set(b) and sorted(a + b) == list(range(16))


def test_lpt_assignment_balances_and_is_deterministic():
    from paper_2408_02758_gb300 import dist as D

    costs = [8, 7, 6, 5, 4, 3, 2, 1]
    bins = D.lpt_assign(costs, 3)
    loads = [sum(costs[i] for i in b) for b in bins]
    assert sorted(sum(bins, [])) == list(range(8))
    assert max(loads) - min(loads) <= 2
    assert D.lpt_assign(costs, 3) == bins
    assert D.lpt_assign(costs, 1) == [list(range(8))]

"""Sharding of the batched form's ensemble over GPUs (one process per GPU):
the placement by longest processing time first on N cap^2, checked on CPU
with two gloo ranks -- every member on exactly one rank, the loads within
Graham's bound, and the gathered cell count counting each member once."""
import os
import socket

import pytest

from paper_2408_03483_gb300 import shard
from synth import ensemble


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws = ensemble(256)
        costs = [shard.member_cost(w["n"], w["cap"]) for w in ws]
        mine = shard.partition(costs, world)[rank]
        cells_mine = sum(ws[i]["n"] ** 2 for i in mine)
        cells = bench.ensemble_cells(cells_mine)
        # every rank's member list, gathered
        t = torch.zeros(256, dtype=torch.int64)
        t[mine] = rank + 1
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        marks = t.tolist()
        cnt = torch.zeros(256, dtype=torch.int64)
        cnt[mine] = 1
        dist.all_reduce(cnt, op=dist.ReduceOp.SUM)
        q.put((rank, cells, marks, cnt.tolist(), mine))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_the_ensemble_exactly():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ws = ensemble(256)
    total = sum(w["n"] ** 2 for w in ws)
    for rank, cells, marks, cnt, mine in out:
        assert cells == total                      # every member's cells, once
        assert cnt == [1] * 256                    # each member on exactly one rank
        assert all(m in (1, 2) for m in marks)
    assert set(out[0][4]).isdisjoint(out[1][4]) and len(out[0][4]) + len(out[1][4]) == 256


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_lpt_loads_within_graham_bound(world):
    ws = ensemble(256)
    costs = [shard.member_cost(w["n"], w["cap"]) for w in ws]
    shards = shard.partition(costs, world)
    assert sorted(i for s in shards for i in s) == list(range(256))
    loads = shard.shard_loads(costs, shards)
    mean = sum(costs) / world
    assert max(loads) <= mean + max(costs) + 1e-9
    # LPT's 4/3 bound against the trivial lower bound max(mean, max cost)
    assert max(loads) <= (4.0 / 3.0) * max(mean, max(costs)) + 1e-9


def test_partition_is_deterministic_and_ties_go_low():
    assert shard.partition([1.0, 1.0, 1.0, 1.0], 2) == [[0, 2], [1, 3]]
    assert shard.partition([5.0, 1.0, 1.0], 2) == [[0], [1, 2]]
    assert shard.partition([], 3) == [[], [], []]
    with pytest.raises(ValueError):
        shard.partition([1.0], 0)

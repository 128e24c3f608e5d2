"""The multi-process (replicas) path of bench.py on CPU: two gloo ranks on
127.0.0.1, each timing its own replica; the job's time is the slowest
rank's, and the throughput counts every rank's units."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, loc = bench.dist_env()
        my_ms = 100.0 + 50.0 * r  # rank 1 is the slow replica
        worst = bench.max_over_ranks(my_ms)
        val = bench.replica_value(1000.0, w, worst)
        dist.barrier()
        q.put((r, w, loc, worst, val))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp
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
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 and o[2] == o[0] for o in out)
    # both ranks agree on the slowest time (150 ms) and on 2000 units / 0.15 s
    assert all(o[3] == pytest.approx(150.0) for o in out)
    assert all(o[4] == pytest.approx(2000.0 / 0.15) for o in out)


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(42.0) == 42.0
    assert bench.replica_value(500.0, 1, 250.0) == pytest.approx(2000.0)

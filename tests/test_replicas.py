"""The N > 1 path of bench.py (independent replicas, one process per GPU):
its host-side aggregation -- barrier, max over ranks, whole-job rate -- run
with world size 2 on the gloo backend (CPU only)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert bench.dist_env() == (rank, world, rank)
        bench.replica_barrier(world)
        local = [1.5, 3.0][rank]            # the second replica is slower
        m = bench.replica_max(local, world)
        rate = bench.replica_throughput(10, local, world)
        out[rank] = (m, rate)
        bench.replica_barrier(world)
    finally:
        dist.destroy_process_group()


def test_replica_aggregation_world2():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    # max over ranks seen identically by both; rate = all units / slowest time
    assert out[0] == out[1] == (3.0, 2 * 10 / 3.0)


def test_single_process_defaults():
    import bench
    assert bench.replica_max(2.5, 1) == 2.5
    assert bench.replica_throughput(4, 2.0, 1) == 2.0

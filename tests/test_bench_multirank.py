"""The benchmark's multi-rank host logic on CPU: two gloo ranks on 127.0.0.1 each
report a local time; the job time is the slowest rank's and the throughput counts
the work of both ranks (weak scaling, one replica per rank)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t_local = 1.0 + rank  # rank 1 is the slow one
    t_max, value = bench.aggregate(t_local, 1e9, 10, world, torch.device("cpu"))
    assert bench._env_rank() == (rank, world, rank)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t_max, value))


def test_two_rank_aggregate_takes_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t_max, value in res:
        assert t_max == pytest.approx(2.0)
        # 2 ranks x 10 steps x 1e9 pairs / 2 s = 10 G pairs/s
        assert value == pytest.approx(10.0)


def test_single_rank_is_local_time():
    import bench
    t, v = bench.aggregate(0.5, 2e9, 4, 1, torch.device("cpu"))
    assert t == 0.5 and v == pytest.approx(16.0)

"""The N > 1 host logic of bench.py on CPU: two gloo ranks, max-over-ranks time
and the whole-job rate (replicas, weak scaling, no data-path collective)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(1.0 + rank)          # rank r took 1 + r seconds
    rate = bench.whole_job_rate(1000, 4, world, t)
    ws, r, local = bench.dist_env()
    out.put((rank, t, rate, ws, r, local))
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_rate():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, rate, ws, r, local in res:
        assert t == 2.0                              # the slowest rank
        assert rate == pytest.approx(1000 * 4 * 2 / 2.0)
        assert (ws, r, local) == (2, rank, rank)


def test_single_process_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.whole_job_rate(10, 2, 1, 4.0) == 5.0

"""The N > 1 path of bench.py on CPU with gloo, world size 2 (no GPU).

Multi-GPU here is replicas only: every rank solves its own instance and the
only collective is the timing reduction (slowest rank).  This checks that
reduction and the whole-job rate with two real processes.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    w, r, local = bench.dist_setup(None)
    assert (w, r, local) == (world, rank, rank)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    my_ms = 100.0 + 50.0 * rank  # rank 1 is the slow one
    ms = bench.max_over_ranks(my_ms, dist, "cpu")
    out[rank] = (ms, bench.whole_job_rate(world, 10, 100, ms / 1e3))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_timing_is_the_slowest_rank():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][0] == res[1][0] == 150.0
    # 2 replicas x 10 steps x 100 iterations in 0.15 s
    assert abs(res[0][1] - 2 * 10 * 100 / 0.15) < 1e-6


def test_single_rank_needs_no_collective():
    import bench

    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5
    assert bench.whole_job_rate(1, 5, 100, 0.5) == 1000.0

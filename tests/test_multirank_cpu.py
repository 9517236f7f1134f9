"""The multi-rank path of bench.py on CPU: two gloo ranks, 127.0.0.1.

Each rank runs its own replica of the workload (no data-path collective); the
only cross-rank step is the maximum of the timed regions, which sets the
whole-job time, and the whole-job rate counts the units of every rank.
"""

import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ws, r, local = bench.dist_env()
    assert (ws, r, local) == (world, rank, rank)
    # rank-dependent step times: the maximum must win on every rank
    got = bench.max_over_ranks([10.0 + rank, 5.0 - rank])
    out[rank] = got
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp

    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == [11.0, 5.0] and out[1] == [11.0, 5.0]


def test_whole_job_rate_counts_every_replica():
    import bench
    assert bench.whole_job_rate(107085, 1, 1000.0) == 107085
    assert bench.whole_job_rate(107085, 4, 2000.0) == 4 * 107085 / 2.0
    assert bench.max_over_ranks([3.0, 4.0]) == [3.0, 4.0]  # no process group: identity

"""The multi-rank path of bench.py on CPU: two gloo ranks (replicas, weak
scaling, max-over-ranks timing, whole-job rate)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist_env()
    assert (r, w, local) == (rank, world, rank)
    my_time = 0.25 + 0.5 * rank                      # rank 1 is the slow one
    t = bench.max_over_ranks(my_time, dist, "cpu")
    rate = bench.whole_job_rate(1 << 20, w, t)
    out[rank] = (t, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn")
    assert out[0] == out[1]
    t, rate = out[0]
    assert t == pytest.approx(0.75)
    assert rate == pytest.approx(2 * (1 << 20) / 0.75 / 1e9)

"""The multi-rank path of bench.py on CPU: two gloo ranks, each its own
replica; the job value is the units of all ranks over the slowest rank's
time (max over ranks), and every rank simulates a different seed."""
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


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    seconds = [2.0, 3.0][rank]
    committed = [100.0, 250.0][rank]
    t_max, value = bench.job_throughput(dist, seconds, committed, "cpu")
    seeds = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(seeds, torch.tensor([bench.replica_seed(rank)], dtype=torch.int64))
    out[rank] = (t_max, value, [int(x.item()) for x in seeds])
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_benchmark():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        t_max, value, seeds = res[rank]
        assert t_max == 3.0
        assert value == pytest.approx(350.0 / 3.0)
        assert len(set(seeds)) == 2


def test_single_rank_needs_no_group():
    import bench
    assert bench.job_throughput(None, 2.0, 10.0, "cpu") == (2.0, 5.0)

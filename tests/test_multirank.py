"""The multi-rank path of bench.py on CPU: two gloo ranks run the benchmark's
own bookkeeping end to end -- each rank draws its own batch (different seeds
per rank), times exactly K steps after W warm-up steps between barriers, and
the job value is the units of all ranks over the slowest rank's time (sum and
max over ranks).  The step here is real work: the oracle simulating two small
lattices of the rank's batch (the GPU step needs a GPU)."""
import os
import socket
import time

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


def _small_lattices(rank):
    import bench
    from paper_cs_0405053_gb300 import workloads
    reps = workloads.batch_replicas(seed0=bench.rank_seed0(rank))
    return [r for r in reps if r["L"] == 64][:2]


def _oracle_step(reps):
    import oracle
    t0 = time.perf_counter()
    c = 0
    for r in reps:
        c += int(oracle.run(r["L"], r["J"], r["h"], r["T"], 16, 16, r["seed"], [1.0],
                            keep_spins=False).counts[-1].sum())
    return time.perf_counter() - t0, c


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    reps = _small_lattices(rank)
    secs, units, wall = bench.timed_steps(lambda: _oracle_step(reps), 3, 1, dist)
    t_max, value = bench.job_throughput(dist, sum(secs), units, "cpu")
    mine = torch.tensor([sum(secs), float(units)], dtype=torch.float64)
    every = [torch.zeros(2, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(every, mine)
    out[rank] = (t_max, value, [tuple(float(v) for v in e) for e in every], len(secs),
                 [r["seed"] for r in reps])
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_run_the_benchmark_bookkeeping():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    per_rank = res[0][2]
    assert res[1][2] == per_rank
    t_max = max(s for s, _ in per_rank)
    total = sum(u for _, u in per_rank)
    for rank in (0, 1):
        got_t, got_v, _, n_steps, seeds = res[rank]
        assert n_steps == 3
        assert got_t == t_max
        assert got_v == pytest.approx(total / t_max)
    # each rank simulated its own lattices; its units are its oracle counts, three steps
    assert set(res[0][4]).isdisjoint(res[1][4])
    for rank in (0, 1):
        _, c = _oracle_step(_small_lattices(rank))
        assert per_rank[rank][1] == 3 * c


def test_single_rank_needs_no_group():
    import bench
    assert bench.job_throughput(None, 2.0, 10.0, "cpu") == (2.0, 5.0)
    secs, units, _ = bench.timed_steps(lambda: (0.5, 7), 4, 3)
    assert secs == [0.5] * 4 and units == 28

"""The benchmark's multi-process logic on CPU ranks (gloo, world size 2):
each rank walks its own batch (distinct seeds and starts), the job's time is
the slowest rank's, and the rate counts the units of all ranks.  The GPU
ranks of a real run use the same helpers over NCCL."""

import os
import socket

import numpy as np
import pytest


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    import bench
    from workloads import gnp_connected, uniform_starts

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    assert bench.dist_env() == (world, rank, rank)
    seed, start_seed = bench.rank_seeds(rank)
    g = gnp_connected(300, 0.05, 1)
    starts = uniform_starts(g, 1000, start_seed)
    # a per-rank "time": rank 1 is the slow one
    mine = 10.0 + 5.0 * rank
    job = bench.max_over_ranks(dist, mine, "cpu")
    rate = bench.whole_job_rate(world, 1000 * 64, job / 1e3)
    dist.barrier()
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), seed=seed, starts=starts, job=job, rate=rate)
    dist.destroy_process_group()


def test_two_rank_sharding_and_timing(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    world = 2
    mp.spawn(rank_main, args=(world, free_port(), str(tmp_path)), nprocs=world, join=True)
    r = [np.load(tmp_path / f"rank{i}.npz") for i in range(world)]
    assert int(r[0]["seed"]) != int(r[1]["seed"])
    assert not np.array_equal(r[0]["starts"], r[1]["starts"])
    for x in r:
        assert float(x["job"]) == 15.0  # max over ranks
        assert float(x["rate"]) == pytest.approx(world * 1000 * 64 / 0.015)


def test_single_process_helpers():
    import bench
    assert bench.max_over_ranks(None, 3.5, "cpu") == 3.5
    assert bench.whole_job_rate(4, 100.0, 2.0) == 200.0
    seeds = {bench.rank_seeds(r) for r in range(8)}
    assert len(seeds) == 8

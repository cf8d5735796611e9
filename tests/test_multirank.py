"""The multi-GPU path of bench.py on CPU: two gloo ranks.  Each rank works on
its own problem (distinct field seeds, no data exchange); the job time is the
maximum over ranks and the throughput counts the units of all ranks."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    local_ms = 100.0 + 50.0 * rank
    job_ms = bench._max_over_ranks(local_ms, dist, device="cpu")
    seeds = [None] * world
    dist.all_gather_object(seeds, bench._rank_seed(rank))
    out[rank] = (job_ms, seeds)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_independent_problems_and_max_time():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        job_ms, seeds = out[r]
        assert job_ms == 150.0
        assert len(set(seeds)) == world
    # whole-job value: seconds per propagator over all ranks' propagators
    steps = 5
    assert (150.0 / 1e3) / (steps * world) == pytest.approx(0.015)

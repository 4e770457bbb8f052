"""The multi-process path of bench.py on the CPU: two gloo ranks.

With N > 1 processes every rank advances its own replica of the workload (independent seeds, no
data-path collective) and the whole-job value is the particle-steps of all ranks over the slowest
rank's time.  These tests run that host logic -- the rank helpers, the replica seeds, the reduction
and the reference arm's "rank 0 alone" rule -- in two gloo processes, without a GPU.
"""
import contextlib
import io
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, out):
    import sys

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ranks = bench.Ranks(dist, "cpu")
        ranks.barrier()
        # rank r processed 1000 * (r + 1) particle-steps in 10 * (r + 1) ms
        value, ms_max = bench.whole_job(1000.0 * (rank + 1), 10.0 * (rank + 1), ranks)
        seed = bench.replica_params("c2", rank)["seed"]
        seeds = [None] * world
        dist.all_gather_object(seeds, seed)

        class Args:
            workload, steps, warmup, gpus = "c1", 1, 1, world

        printed = io.StringIO()
        if rank != 0:
            with contextlib.redirect_stdout(printed):
                bench.run_reference(Args, rank, world)
        out.put((rank, value, ms_max, seeds, printed.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_and_seed_replicas():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    try:
        for _ in range(world):
            rank, value, ms_max, seeds, printed = out.get(timeout=120)
            res[rank] = (value, ms_max, seeds, printed)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    # whole job: (1000 + 2000) particle-steps over the slowest rank's 20 ms, the same on every rank
    for r in range(world):
        value, ms_max, seeds, printed = res[r]
        assert ms_max == 20.0
        assert value == pytest.approx(3000.0 / 0.020, rel=1e-15)
        assert len(set(seeds)) == world  # each replica draws its own particles and collisions
    # the reference arm: ranks other than 0 print nothing and do no work
    assert res[1][3] == ""


def test_lone_process_needs_no_process_group():
    import sys

    sys.path.insert(0, ROOT)
    import bench

    ranks = bench.Ranks(None, "cpu")
    ranks.barrier()
    assert bench.whole_job(5.0e6, 2.5, ranks) == (5.0e6 / 0.0025, 2.5)
    assert bench.replica_params("c3", 0) == bench.W.CONFIGS["c3"]

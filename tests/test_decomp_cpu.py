"""Host side of the particle decomposition on two gloo ranks (CPU): the deposit exchange is an
exact int64 sum over the ranks -- no rounding even near the int64 range, whatever the order -- and
the id rule of pic_keep_subset (id % nparts == part) gives every particle to exactly one part."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist

    from paper_2606_28534_gb300 import decomp

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    assert decomp.rank_and_size() == (rank, world)
    big = (1 << 61) + 12345  # sums beyond 2^53: a float reduction would round them
    R = torch.tensor([big * (rank + 1), -3 * rank, rank], dtype=torch.int64)
    decomp.exchange(R)
    out.put((rank, R.tolist()))
    dist.destroy_process_group()


def test_deposit_exchange_is_an_exact_int64_sum_on_two_gloo_ranks():
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    big = (1 << 61) + 12345
    want = [big * 3, -3, 1]
    assert got[0] == want and got[1] == want


def test_exchange_without_a_process_group_leaves_the_deposits():
    import torch

    from paper_2606_28534_gb300 import decomp

    R = torch.arange(6, dtype=torch.int64)
    assert decomp.rank_and_size() == (0, 1)
    assert decomp.exchange(R).tolist() == list(range(6))


@pytest.mark.parametrize("nparts", [1, 2, 3, 7])
def test_the_id_rule_partitions_every_kind_of_id(nparts):
    # load ids (electrons i, ions 2^62 | i), pair-source ids 2^63 | ..., random 64-bit child ids
    rng = np.random.default_rng(4)
    ids = np.concatenate([np.arange(1000, dtype=np.uint64), (np.uint64(1) << np.uint64(62)) | np.arange(1000, dtype=np.uint64),
                          rng.integers(0, 2**63, 1000, dtype=np.uint64) | np.uint64(1 << 63)])
    owner = ids % np.uint64(nparts)
    counts = np.bincount(owner.astype(np.int64), minlength=nparts)
    assert counts.sum() == len(ids) and (owner < nparts).all()
    if nparts > 1:
        assert counts.min() > 0.8 * len(ids) / nparts  # a balanced split of the load's ids

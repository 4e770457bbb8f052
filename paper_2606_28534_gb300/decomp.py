"""Particle decomposition of one simulation over the ranks of a torch.distributed process group.

The paper spreads one simulation over many GPUs by MPI domain decomposition with particle load
balancing (Sec. 4.1).  Here every rank keeps a subset of the particles (ids with id % world ==
rank) over the whole grid, and the ranks exchange one thing per step: their int64 node deposits,
summed by an all-reduce.  The sum of integers is exact in any order, so every rank solves the same
field and the union of the ranks' particles evolves exactly as one simulation holding them all.
Every step of the method runs in the library's kernels (pic_step_begin / pic_step_end); this
module only moves the deposit tensor between the calls.
"""
from __future__ import annotations

from . import pic


def exchange(R, group=None):
    """Sum the int64 node deposits R over the ranks of group, in place.  NCCL reduces the CUDA
    tensor itself; other backends (gloo) reduce a host copy.  With one rank (or no process group)
    R is left as it is."""
    import torch.distributed as dist

    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size(group) == 1:
        return R
    if dist.get_backend(group) == "nccl":
        dist.all_reduce(R, op=dist.ReduceOp.SUM, group=group)
        return R
    host = R.cpu()
    dist.all_reduce(host, op=dist.ReduceOp.SUM, group=group)
    R.copy_(host)
    return R


def rank_and_size(group=None):
    import torch.distributed as dist

    if not dist.is_available() or not dist.is_initialized():
        return 0, 1
    return dist.get_rank(group), dist.get_world_size(group)


class Decomposed:
    """This rank's part of one simulation decomposed by particles.  Every rank constructs it with
    the same parameters; step() advances all parts together (it is collective)."""

    def __init__(self, params: dict, group=None, device=None, stream=None):
        import torch

        self.group = group
        self.rank, self.world = rank_and_size(group)
        self.sim = pic.Simulation(params, device=device, stream=stream)
        self.sim.keep_subset(self.rank, self.world)
        self.R = torch.empty(2 * (self.sim.N + 1), dtype=torch.int64, device=self.sim.device)
        with torch.cuda.stream(self.sim.stream):
            self.sim.local_deposit(self.R)
            exchange(self.R, group)
            self.sim.solve_deposit(self.R)

    def step(self, n: int = 1):
        import torch

        with torch.cuda.stream(self.sim.stream):
            for _ in range(int(n)):
                self.sim.step_begin(self.R)
                exchange(self.R, self.group)
                self.sim.step_end(self.R)

    def close(self):
        self.sim.close()

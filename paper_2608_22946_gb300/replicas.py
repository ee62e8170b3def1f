"""Replica multi-GPU use of the solver: one process per GPU, each solving its
own share of the independent right-hand sides (point sources) of one
frequency and velocity model.  Sources share nothing but the read-only
model, so the data path has no collective; the adjoint-state gradient of the
receiver misfit is a sum over sources, whose only exchange is one all-reduce
of the N_h gradient (and of the scalar misfit).

The helpers are host logic around ``torch.distributed`` (NCCL on GPUs, gloo
on the host); every solve runs in the library's kernels.
"""
from __future__ import annotations


def partition(n: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous, balanced share [start, stop) of n items for `rank` of
    `world` (the first n % world ranks take one more)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    q, r = divmod(n, world)
    start = rank * q + min(rank, r)
    return start, start + q + (1 if rank < r else 0)


def allreduce_sum(t, pg=None):
    """Sum a tensor over the ranks of the default process group (in place;
    returned).  A no-op without a process group."""
    import torch.distributed as dist
    if pg is None and not (dist.is_available() and dist.is_initialized()):
        return t
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=pg)
    return t


def sharded_misfit_gradient(misfit_grad, sources, d_obs, world: int = 1, rank: int = 0, pg=None):
    """Misfit and gradient summed over all sources, each rank evaluating its
    share.  misfit_grad(sources_subset, d_obs_subset) -> (J, g) with g a
    torch tensor (the rank's device); d_obs has one row per source.  Returns
    (J, g) summed over ranks on every rank."""
    import torch
    a, b = partition(len(sources), world, rank)
    if b > a:
        J, g = misfit_grad(list(sources[a:b]), d_obs[a:b])
        J = torch.tensor([float(J)], dtype=torch.float64, device=g.device)
    else:
        raise ValueError("more ranks than sources: every rank needs at least one source")
    allreduce_sum(g, pg)
    allreduce_sum(J, pg)
    return float(J.item()), g

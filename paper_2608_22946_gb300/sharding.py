"""Spatial sharding of the fine level as z-slab bricks: the decomposition of
the paper's multi-GPU runs (Sec. 6.1: bricks with a one-node halo exchanged
with the neighbours before each stencil application, and an all-reduce for
every Krylov inner product), in the one-axis form.

Each rank owns planes [z0, z1) of every fine-level field.  Before an operator
application it receives the plane just below and just above its slab from the
neighbouring ranks (zeros at the ends of the grid), and the library applies
the operator to its rows from that window (``Solver.iofd_apply_window``);
every row then takes exactly the arithmetic of the unsharded application.
Inner products are local partial sums combined by one all-reduce.

The helpers are host logic around ``torch.distributed`` (NCCL between GPUs,
gloo on the host); the operator itself runs in the library's kernels.
"""
from __future__ import annotations

from .replicas import partition


def slab(nz: int, world: int, rank: int) -> tuple[int, int]:
    """Planes [z0, z1) of the fine level owned by `rank` of `world` (balanced)."""
    if nz < world:
        raise ValueError("fewer planes than ranks")
    return partition(nz, world, rank)


def _dist():
    import torch.distributed as dist
    return dist if (dist.is_available() and dist.is_initialized()) else None


def halo_window(local, world: int, rank: int, pg=None):
    """The window of an operator application for a rank's slab.

    local: tensor (nrhs, nzl, ny, nx), the rank's planes.  Returns
    (nrhs, nzl + 2, ny, nx): the plane below from rank - 1, the slab, the
    plane above from rank + 1, and zeros where the slab ends at the grid.
    Uses blocking send/receive with the neighbours (every rank calls it)."""
    import torch
    nrhs, nzl = local.shape[0], local.shape[1]
    win = torch.zeros((nrhs, nzl + 2) + tuple(local.shape[2:]), dtype=local.dtype, device=local.device)
    win[:, 1:nzl + 1] = local
    dist = _dist()
    if world == 1 or dist is None:
        return win
    # complex planes travel as real pairs (not every backend carries complex)
    real = (lambda t: torch.view_as_real(t.contiguous())) if local.is_complex() else (lambda t: t.contiguous())
    below = torch.empty_like(real(local[:, 0]))
    above = torch.empty_like(below)
    reqs = []
    if rank > 0:
        reqs.append(dist.isend(real(local[:, 0]), rank - 1, group=pg))
        reqs.append(dist.irecv(below, rank - 1, group=pg))
    if rank < world - 1:
        reqs.append(dist.isend(real(local[:, nzl - 1]), rank + 1, group=pg))
        reqs.append(dist.irecv(above, rank + 1, group=pg))
    for req in reqs:
        req.wait()
    back = (lambda t: torch.view_as_complex(t)) if local.is_complex() else (lambda t: t)
    if rank > 0:
        win[:, 0] = back(below)
    if rank < world - 1:
        win[:, nzl + 1] = back(above)
    return win


def sharded_apply(apply_window, local, z0: int, z1: int, world: int, rank: int, pg=None):
    """Rows [z0, z1) of Op x for the rank's slab: halo exchange, then
    apply_window(window, z0, z1) (e.g. ``Solver.iofd_apply_window``)."""
    return apply_window(halo_window(local, world, rank, pg), z0, z1)


def sharded_dot(a, b, pg=None):
    """Per right-hand side sum over all ranks of conj(a) . b (complex128 on the
    host side of the reduction), one all-reduce."""
    import torch
    part = (a.conj() * b).reshape(a.shape[0], -1).sum(dim=1).to(torch.complex128)
    dist = _dist()
    if dist is None:
        return part
    buf = torch.view_as_real(part).contiguous()
    dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=pg)
    return torch.view_as_complex(buf)

"""Column-block partition of the full reduced Hessian over several ranks.

Section 5.3 computes H = (Hess F) I block by block; the blocks of columns are
independent once every rank holds the per-state data (factors, lambda,
projection coefficients).  Rank r of `world` computes the contiguous columns
``column_range(n_p, world, r)`` with ``rh_hessian_columns``; one gather then
puts the blocks, in column order, into the destination rank's H.  Nothing
else is exchanged.

The gather goes through ``torch.distributed`` on whatever backend the process
group has (gloo with CPU tensors, NCCL with CUDA tensors).
"""
from __future__ import annotations

import numpy as np


def column_range(n_p: int, world: int, rank: int) -> tuple[int, int]:
    """(first column, number of columns) of rank's block: contiguous, sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must be in [0, world)")
    c0 = rank * n_p // world
    c1 = (rank + 1) * n_p // world
    return c0, c1 - c0


def local_block(grid, world: int, rank: int, out=None, stream=None):
    """This rank's columns of H on its grid (an adjoint-ready ``rh.Grid``): a numpy array, or
    ``out`` (a column-major CUDA tensor of n_p x ncols) when given."""
    c0, n = column_range(grid.n_p, world, rank)
    return grid.hessian_columns(c0, n, out=out, stream=stream)


def gather_columns(block, n_p: int, world: int, rank: int, dst: int = 0, group=None):
    """Gather every rank's (n_p x ncols) block into the full n_p x n_p H on rank ``dst``.

    ``block`` is this rank's block (numpy array or torch tensor; a CUDA tensor for NCCL).
    Returns H on ``dst`` (same kind as ``block``: column-major numpy, or a torch tensor
    of shape (n_p, n_p) whose column j is H[:, j]) and None on the other ranks.
    Blocks are padded to the widest one for the collective and trimmed after it.
    """
    import torch
    import torch.distributed as dist

    is_np = isinstance(block, np.ndarray)
    t = torch.from_numpy(np.ascontiguousarray(np.asarray(block).T)) if is_np else block.t().contiguous()
    width = -(-n_p // world)
    _, n = column_range(n_p, world, rank)
    if t.shape[0] != n or t.shape[1] != n_p:
        raise ValueError("block does not match this rank's column range")
    pad = torch.zeros((width, n_p), dtype=t.dtype, device=t.device)
    pad[:n] = t
    parts = [torch.empty_like(pad) for _ in range(world)] if rank == dst else None
    dist.gather(pad, gather_list=parts, dst=dst, group=group)
    if rank != dst:
        return None
    rows = torch.cat([parts[r][:column_range(n_p, world, r)[1]] for r in range(world)], dim=0)   # (n_p cols, n_p)
    if is_np:
        return np.asfortranarray(rows.numpy().T)
    return rows.t()

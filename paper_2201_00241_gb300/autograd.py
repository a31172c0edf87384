"""The reduced objective F(p) = f(x(p), p) of Eq. 5 as a torch.autograd.Function.

forward:          F(p)    device Newton power flow at p, then rh_adjoint
backward:         grad F  the first-order adjoint, Eq. 7
double backward:  H w     the reduced-Hessian-vector product, Eq. 9-10 (rh_hessvec)

All numerical work runs in librh's kernels; these classes only move arguments.
With p on a CUDA device the products stay there: rh_hessvec reads w and writes
H w in device memory on the current stream, with no host round trip.  A block
of directions (several grad_outputs) is one rh_hessvec launch through
``reduced_hessian_vector_products``.
The library grid is stateful (its loads, x and factors), so every evaluation
first makes sure the grid's state is the one at the requested p.
"""
from __future__ import annotations

import numpy as np
import torch


def _ensure_state(grid, p: torch.Tensor, x0=None, tol: float = 1e-13, max_iter: int = 20):
    """Set the parameters p on the grid, re-solve the power flow and the adjoint if p changed."""
    pn = np.ascontiguousarray(p.detach().to("cpu", torch.float64).numpy())
    key = pn.tobytes()
    if getattr(grid, "_ad_key", None) == key:
        return
    grid.set_state(pn)
    start = x0 if x0 is not None else getattr(grid, "_ad_x", None)
    x, _, _, _ = grid.powerflow(start, tol=tol, max_iter=max_iter)
    lam, grad, F = grid.adjoint()
    grid._ad_key, grid._ad_x, grid._ad_grad, grid._ad_F = key, x, grad, F


def _hessvec_block(grid, W: torch.Tensor, like: torch.Tensor) -> torch.Tensor:
    """H W for an (n_p, N) block in one rh_hessvec call, on the device of `like`:
    device pointers on the current stream for CUDA tensors, host buffers otherwise."""
    if like.is_cuda:
        Wc = W.detach().to(device=like.device, dtype=torch.float64)
        Wc = Wc.t().contiguous().t()                  # column-major n_p x N
        return grid.hessvec(Wc)
    hw = grid.hessvec(np.asfortranarray(W.detach().to("cpu", torch.float64).numpy()))
    return torch.as_tensor(hw, dtype=torch.float64)


class _ReducedGradient(torch.autograd.Function):
    @staticmethod
    def forward(ctx, p, grid):
        _ensure_state(grid, p)
        ctx.grid = grid
        ctx.save_for_backward(p)
        return torch.as_tensor(grid._ad_grad, dtype=torch.float64, device=p.device).clone()

    @staticmethod
    def backward(ctx, v):
        (p,) = ctx.saved_tensors
        grid = ctx.grid
        _ensure_state(grid, p)
        hw = _hessvec_block(grid, v.reshape(-1, 1), p)[:, 0]   # H is symmetric: v^T H = (H v)^T
        return hw, None


class ReducedObjective(torch.autograd.Function):
    """F(p) for a library grid whose loads are already set (rh_set_state).

    Use ``reduced_objective(p, grid)``; p is a float64 tensor of length n_p."""

    @staticmethod
    def forward(ctx, p, grid):
        _ensure_state(grid, p)
        ctx.grid = grid
        ctx.save_for_backward(p)
        return torch.tensor(grid._ad_F, dtype=torch.float64, device=p.device)

    @staticmethod
    def backward(ctx, gF):
        (p,) = ctx.saved_tensors
        g = _ReducedGradient.apply(p, ctx.grid)
        return gF * g, None


def reduced_objective(p: torch.Tensor, grid) -> torch.Tensor:
    return ReducedObjective.apply(p, grid)


def reduced_hessian_vector_products(p: torch.Tensor, grid, W: torch.Tensor) -> torch.Tensor:
    """(Hess F)(p) W for a block of directions W (n_p x N, float64) in one rh_hessvec
    launch: what N separate grad_outputs of the gradient would give, column by column.
    On the device of p (device pointers, the current stream) or on the host.  Not
    differentiable further: third derivatives are not provided."""
    _ensure_state(grid, p)
    return _hessvec_block(grid, W, p)

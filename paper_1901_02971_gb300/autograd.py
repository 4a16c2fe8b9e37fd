"""Differentiable spaND solve: x = A(vals)^{-1} b as a torch.autograd.Function.

Forward: factorize A (if its values changed) and run PCG through the C ABI.
Backward (A is SPD, so the adjoint system is the same system):
    lam   = A^{-1} dL/dx        (a second PCG solve with the same factorization)
    dL/db = lam
    dL/dA = -lam x^T restricted to A's stored pattern (spand_sampled_outer),
            one value per stored entry, in the CSR order of the values.
All arithmetic runs in libspand.so kernels; this module only marshals tensors.
"""
from __future__ import annotations

import torch

from . import _lib as L
from .solver import Solver


class SpandSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vals: torch.Tensor, b: torch.Tensor, solver: Solver):
        vals = vals.detach().contiguous()
        if not (vals.is_cuda and vals.dtype == torch.float64):
            raise ValueError("vals must be a float64 CUDA tensor")
        if getattr(solver, "_vals_version", None) is not vals or getattr(solver, "_vals_stamp", None) != vals._version:
            solver.factorize(vals)
            solver._vals_version = vals
            solver._vals_stamp = vals._version
        b = b.detach().contiguous()
        x = torch.empty_like(b)
        solver.solve(b, x)
        ctx.solver = solver
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, gx: torch.Tensor):
        (x,) = ctx.saved_tensors
        solver = ctx.solver
        gx = gx.detach().contiguous().to(torch.float64)
        lam = torch.empty_like(gx)
        if torch.count_nonzero(gx) == 0:
            lam.zero_()
        else:
            solver.solve(gx, lam)
        gvals = None
        if ctx.needs_input_grad[0]:
            gvals = torch.empty(int(solver.nnz), dtype=torch.float64, device=x.device)
            L.spand_sampled_outer(solver.h, lam.data_ptr(), x.data_ptr(), gvals.data_ptr(),
                                  torch.cuda.current_stream().cuda_stream)
        gb = lam if ctx.needs_input_grad[1] else None
        return gvals, gb, None


def spand_solve(vals: torch.Tensor, b: torch.Tensor, solver: Solver) -> torch.Tensor:
    """x = A(vals)^{-1} b, differentiable with respect to vals and b."""
    return SpandSolve.apply(vals, b, solver)

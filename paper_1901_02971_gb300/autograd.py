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


class CoefficientAssembly:
    """Differentiable map from a cell coefficient field a to the stored values
    of A = -div(a grad .) on a 2D or 3D grid (5- / 7-point stencil, Dirichlet
    faces), for gradients with respect to a (the batch of diffusion problems
    of the benchmark's differentiable form).

    Same discretisation as the problem generators: the face between cells i
    and j carries f_ij = 2 a_i a_j / (a_i + a_j) (harmonic mean), giving
    A_ij = A_ji = -f_ij and adding f_ij to A_ii and A_jj; a face on the
    Dirichlet boundary adds the cell's own a_i to A_ii; no h^2 scaling.  The
    CSR pattern (rowptr, colind: the generator's, x fastest) is fixed; the
    values come out in its order, so that dL/dvals from the solve chains
    into dL/da by torch autograd.

    shape: grid shape in numpy order ((ny, nx) or (nz, ny, nx)).
    """

    def __init__(self, shape, rowptr, colind, device="cuda"):
        import numpy as np
        self.shape = tuple(int(v) for v in shape)
        dim = len(self.shape)
        n = int(np.prod(self.shape))
        rowptr = np.asarray(rowptr, dtype=np.int64)
        colind = np.asarray(colind, dtype=np.int64)
        rows = np.repeat(np.arange(n), np.diff(rowptr))
        ids = np.arange(n).reshape(self.shape)
        # face lists per grid axis (x first): lower cell i0, upper cell i1;
        # face_of[ax][i0] = index of that face among [diag | faces of axis 0 | ...]
        self.faces = []
        face_of = []
        strides = []
        base = n
        for ax in range(dim):
            nax = dim - 1 - ax
            lo = [slice(None)] * dim
            hi = [slice(None)] * dim
            lo[nax] = slice(0, -1)
            hi[nax] = slice(1, None)
            i0, i1 = ids[tuple(lo)].ravel(), ids[tuple(hi)].ravel()
            self.faces.append((torch.as_tensor(i0, device=device), torch.as_tensor(i1, device=device)))
            fo = np.full(n, -1, dtype=np.int64)
            fo[i0] = base + np.arange(i0.size)
            face_of.append(fo)
            strides.append(int(np.prod(self.shape[nax + 1:])))
            base += i0.size
        # boundary faces per axis: cells on the first and last layer
        self.bnd = []
        for ax in range(dim):
            nax = dim - 1 - ax
            first = [slice(None)] * dim
            last = [slice(None)] * dim
            first[nax] = 0
            last[nax] = -1
            self.bnd.append(torch.as_tensor(np.concatenate([ids[tuple(first)].ravel(), ids[tuple(last)].ravel()]),
                                            device=device))
        # every stored entry: the diagonal of its row (index r) or minus the
        # coefficient of its face (index n + face number)
        src = rows.copy()
        lo, d = np.minimum(rows, colind), np.abs(rows - colind)
        for ax in range(dim):
            m = d == strides[ax]
            src[m] = face_of[ax][lo[m]]
        if np.any((d != 0) & (src < n)) or np.any(src < 0):
            raise ValueError("pattern is not the stencil of this grid")
        self.src = torch.as_tensor(src, device=device)
        self.sign = torch.as_tensor(np.where(rows == colind, 1.0, -1.0), device=device)
        self.n = n

    def __call__(self, a: torch.Tensor) -> torch.Tensor:
        a = a.reshape(-1)
        fs = [2.0 * a[i0] * a[i1] / (a[i0] + a[i1]) for i0, i1 in self.faces]
        diag = torch.zeros(self.n, dtype=a.dtype, device=a.device)
        for (i0, i1), f in zip(self.faces, fs):
            diag = diag.index_add(0, i0, f).index_add(0, i1, f)
        for cells in self.bnd:
            diag = diag.index_add(0, cells, a[cells])
        allv = torch.cat([diag] + fs)
        return allv[self.src] * self.sign

"""Differentiable solve (torch.autograd.Function around spand_solve).

dL/db = A^{-1} dL/dx and dL/dA = -lam x^T on A's pattern, with lam from the
adjoint solve that reuses the factorization.  Checked against a dense FP64
reference (numpy) and against central finite differences of the loss with
respect to symmetric pairs of stored values (A must stay symmetric for PCG).
"""
import numpy as np
import pytest

from paper_1901_02971_gb300 import Solver
from paper_1901_02971_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _setup(n=20, seed=3):
    import torch
    p = I.diffusion_2d(n, seed)
    s = Solver.from_problem(p, levels=5, eps=1e-2, tol=1e-12)
    vals = torch.from_numpy(p.vals.copy()).cuda()
    b = torch.from_numpy(I.rhs(p.n, 7)).cuda()
    xstar = torch.from_numpy(I.rhs(p.n, 8)).cuda()
    return p, s, vals, b, xstar


def _loss(vals, b, xstar, s):
    from paper_1901_02971_gb300.autograd import spand_solve
    x = spand_solve(vals, b, s)
    return ((x - xstar) ** 2).sum()


def test_gradients_match_dense_reference(cuda_ok):
    import torch
    p, s, vals, b, xstar = _setup()
    try:
        v = vals.clone().requires_grad_(True)
        bb = b.clone().requires_grad_(True)
        loss = _loss(v, bb, xstar, s)
        loss.backward()
        A = p.to_scipy().toarray()
        x = np.linalg.solve(A, b.cpu().numpy())
        gx = 2 * (x - xstar.cpu().numpy())
        lam = np.linalg.solve(A, gx)
        rows = np.repeat(np.arange(p.n), np.diff(p.rowptr))
        g_ref = -lam[rows] * x[p.colind]
        assert np.linalg.norm(bb.grad.cpu().numpy() - lam) <= 1e-8 * np.linalg.norm(lam)
        assert np.linalg.norm(v.grad.cpu().numpy() - g_ref) <= 1e-8 * np.linalg.norm(g_ref)
    finally:
        s.close()


def test_gradients_match_finite_differences(cuda_ok):
    import torch
    p, s, vals, b, xstar = _setup(n=16, seed=5)
    try:
        v = vals.clone().requires_grad_(True)
        loss = _loss(v, b, xstar, s)
        loss.backward()
        g = v.grad.cpu().numpy()
        rows = np.repeat(np.arange(p.n), np.diff(p.rowptr))
        rng = I.rng(11)
        picks = rng.choice(p.nnz, size=8, replace=False)
        for e in picks:
            i, j = int(rows[e]), int(p.colind[e])
            et = int(np.flatnonzero((rows == j) & (p.colind == i))[0])
            pair = {e, et}
            h = 1e-6 * abs(float(p.vals[e]))
            def f(sign):
                w = vals.clone()
                for q in pair:
                    w[q] += sign * h
                with torch.no_grad():
                    return float(_loss(w, b, xstar, s))
            fd = (f(+1) - f(-1)) / (2 * h)
            an = sum(float(g[q]) for q in pair)
            assert abs(fd - an) <= 1e-5 * max(1.0, abs(an)), (e, fd, an)
    finally:
        s.close()

"""Batches of independent systems: spand_analyze_batch, then concurrent
factorizations and solves (one CUDA stream and one host thread per system).

* A batch run gives bit for bit the results of running each system alone:
  every kernel is deterministic and independent handles share no device data.
* The batch of 32 2D diffusion problems (128^2 ... 512^2 cells, log-normal
  coefficients) converges to the requested residual, each system checked on
  the host against its own matrix.
* Gradients of a loss summed over a batch match a dense FP64 reference.
"""
import numpy as np
import pytest

from paper_1901_02971_gb300 import Solver, factorize_all, solve_all
from paper_1901_02971_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _small_batch(k=6):
    probs, opts = [], []
    for i in range(k):
        p = I.diffusion_2d(24 + 8 * i, 40 + i)
        probs.append(p)
        opts.append(dict(levels=int(round(np.log2(p.n / 32))) + 1, eps=1e-2, precision="fp32", tol=1e-10))
    return probs, opts


def test_batch_concurrent_equals_sequential(cuda_ok):
    import torch
    probs, opts = _small_batch()
    bs = [torch.from_numpy(I.rhs(p.n, 7 + i)).cuda() for i, p in enumerate(probs)]
    batch = Solver.batch(probs, opts)
    alone = [Solver.from_problem(p, **o) for p, o in zip(probs, opts)]
    try:
        factorize_all(batch)
        res = solve_all(batch, bs)
        for s, b, (x, it, rr) in zip(alone, bs, res):
            s.factorize()
            x1, it1, rr1 = s.solve(b)
            torch.cuda.synchronize()
            assert it == it1 and rr == rr1
            assert torch.equal(x, x1)
            assert rr <= 1e-10
    finally:
        for s in batch + alone:
            s.close()


def test_batch_32_diffusion_problems(cuda_ok):
    import torch
    items = [I.batch_diffusion_2d(i) for i in range(32)]
    probs = [it[0] for it in items]
    assert sum(p.n for p in probs) > 3_600_000
    opts = [dict(levels=it[3], eps=1e-2, precision="fp32", tol=1e-10) for it in items]
    solvers = Solver.batch(probs, opts)
    try:
        factorize_all(solvers)
        bs = [torch.from_numpy(it[2]).cuda() for it in items]
        res = solve_all(solvers, bs)
        for (p, xs, b, lv), (x, it, rr) in zip(items, res):
            xh = x.cpu().numpy()
            true_rr = np.linalg.norm(b - p.to_scipy() @ xh) / np.linalg.norm(b)
            assert rr <= 1e-10 and true_rr <= 1.5e-10, (p.name, it, rr, true_rr)
            assert it <= 40, (p.name, it)
            assert np.linalg.norm(xh - xs) <= 1e-6 * np.linalg.norm(xs), p.name
    finally:
        for s in solvers:
            s.close()


def test_batch_gradients_match_dense(cuda_ok):
    """loss = sum_i ||x_i - y_i||^2, x_i = A_i(vals_i)^{-1} b_i, with targets
    y_i independent of b_i (with b_i = A_i x*_i and y_i = x*_i the loss would
    sit at its minimum and every gradient vanish)."""
    import torch
    from paper_1901_02971_gb300.autograd import spand_solve
    probs, opts = _small_batch(3)
    opts = [dict(o, precision="fp64", tol=1e-12) for o in opts]
    solvers = Solver.batch(probs, opts)
    try:
        vals = [torch.from_numpy(p.vals.copy()).cuda().requires_grad_(True) for p in probs]
        bs = [torch.from_numpy(I.rhs(p.n, 60 + i)).cuda().requires_grad_(True) for i, p in enumerate(probs)]
        ys = [torch.from_numpy(I.rhs(p.n, 80 + i)).cuda() for i, p in enumerate(probs)]
        loss = sum(((spand_solve(v, b, s) - y) ** 2).sum() for v, b, s, y in zip(vals, bs, solvers, ys))
        loss.backward()
        for p, v, b, y in zip(probs, vals, bs, ys):
            A = p.to_scipy().toarray()
            x = np.linalg.solve(A, b.detach().cpu().numpy())
            lam = np.linalg.solve(A, 2 * (x - y.cpu().numpy()))
            rows = np.repeat(np.arange(p.n), np.diff(p.rowptr))
            g_ref = -lam[rows] * x[p.colind]
            assert np.linalg.norm(b.grad.cpu().numpy() - lam) <= 1e-8 * np.linalg.norm(lam)
            assert np.linalg.norm(v.grad.cpu().numpy() - g_ref) <= 1e-8 * np.linalg.norm(g_ref)
    finally:
        for s in solvers:
            s.close()

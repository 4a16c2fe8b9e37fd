"""Gradients with respect to the coefficient field a and the right-hand side
b (the differentiable batch form): x_i = A_i(a_i)^{-1} b_i through
spand_solve (adjoint solve on the same factorization, sampled -lam x^T
kernel for dL/dA on A's pattern), chained into dL/da by torch autograd
through the harmonic-mean face assembly.

* a 16^2 instance against a dense FP64 reference (torch.linalg.solve on the
  host, same assembly);
* the batch of 32 problems (128^2 .. 512^2 cells, log-normal a): central
  finite differences on 8 coordinates of a and 8 of b, each in a different
  problem of the batch.

Targets y_i = x*_i + 0.01 xi_i (xi_i ~ N(0, 1)): with y_i = x*_i exactly the
loss would sit at its minimum (b_i = A_i x*_i) and every gradient vanish.
"""
import numpy as np
import pytest

from paper_1901_02971_gb300 import Solver
from paper_1901_02971_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _cells(n, seed):
    return np.exp(I.rng(seed).standard_normal((n, n)))  # the batch generator's field


def test_grad_wrt_a_matches_dense_reference_16x16(cuda_ok):
    import torch
    from paper_1901_02971_gb300.autograd import CoefficientAssembly, spand_solve
    n = 16
    p = I.diffusion_2d(n, 4)
    a0 = torch.from_numpy(_cells(n, 4)).reshape(-1)
    b0 = torch.from_numpy(I.rhs(p.n, 5))
    y = torch.from_numpy(I.rhs(p.n, 6))
    s = Solver.from_problem(p, levels=4, eps=1e-2, tol=1e-13)
    try:
        asm = CoefficientAssembly((n, n), p.rowptr, p.colind, device="cuda")
        a = a0.cuda().requires_grad_(True)
        b = b0.cuda().requires_grad_(True)
        loss = ((spand_solve(asm(a), b, s) - y.cuda()) ** 2).sum()
        loss.backward()
        # dense FP64 reference through the same assembly
        asm_h = CoefficientAssembly((n, n), p.rowptr, p.colind, device="cpu")
        ar = a0.clone().requires_grad_(True)
        br = b0.clone().requires_grad_(True)
        rows = torch.from_numpy(np.repeat(np.arange(p.n), np.diff(p.rowptr)))
        cols = torch.from_numpy(p.colind.astype(np.int64))
        A = torch.zeros(p.n, p.n, dtype=torch.float64).index_put((rows, cols), asm_h(ar))
        lr = ((torch.linalg.solve(A, br) - y) ** 2).sum()
        lr.backward()
        assert abs(float(loss) - float(lr)) <= 1e-9 * float(lr)
        ga, gb = a.grad.cpu(), b.grad.cpu()
        assert float((ga - ar.grad).norm()) <= 1e-8 * float(ar.grad.norm())
        assert float((gb - br.grad).norm()) <= 1e-8 * float(br.grad.norm())
    finally:
        s.close()


def test_batch_32_gradients_match_finite_differences(cuda_ok):
    import torch
    from paper_1901_02971_gb300 import factorize_all
    from paper_1901_02971_gb300.autograd import CoefficientAssembly, spand_solve
    items = [I.batch_diffusion_2d(i) for i in range(32)]
    probs = [it[0] for it in items]
    opts = [dict(levels=it[3], eps=1e-2, precision="fp64", tol=1e-13) for it in items]
    solvers = Solver.batch(probs, opts)
    try:
        n_side = [int(round(np.sqrt(p.n))) for p in probs]
        asms = [CoefficientAssembly((m, m), p.rowptr, p.colind, device="cuda") for m, p in zip(n_side, probs)]
        a0 = [torch.from_numpy(_cells(m, 4 + i)).reshape(-1).cuda() for i, m in enumerate(n_side)]
        b0 = [torch.from_numpy(it[2]).cuda() for it in items]
        ys = [torch.from_numpy(it[1] + 0.01 * I.rhs(p.n, 200 + i)).cuda() for i, (it, p) in enumerate(zip(items, probs))]
        for s, asm, a in zip(solvers, asms, a0):  # the assembled values are the generator's
            s._vals0 = asm(a).detach()
        factorize_all(solvers, [s._vals0 for s in solvers])
        av = [a.clone().requires_grad_(True) for a in a0]
        bv = [b.clone().requires_grad_(True) for b in b0]
        loss = sum(((spand_solve(asm(a), b, s) - y) ** 2).sum() for asm, a, b, s, y in zip(asms, av, bv, solvers, ys))
        loss.backward()

        def loss_i(i, a, b):
            with torch.no_grad():
                x = spand_solve(asms[i](a), b, solvers[i])
                return float(((x - ys[i]) ** 2).sum())

        rng = I.rng(77)
        picked = [0, 5, 10, 15, 20, 25, 30, 31]
        for i in picked:  # one coefficient of a per problem
            k = int(rng.integers(probs[i].n))
            h = 1e-5 * float(a0[i][k])
            ap, am = a0[i].clone(), a0[i].clone()
            ap[k] += h
            am[k] -= h
            fd = (loss_i(i, ap, b0[i]) - loss_i(i, am, b0[i])) / (2 * h)
            an = float(av[i].grad[k])
            assert abs(fd - an) <= 1e-4 * abs(an) + 1e-7 * float(av[i].grad.abs().max()), (i, k, fd, an)
        for i in picked:  # one entry of b per problem (the loss is quadratic in b)
            k = int(rng.integers(probs[i].n))
            h = 1e-3
            bp, bm = b0[i].clone(), b0[i].clone()
            bp[k] += h
            bm[k] -= h
            fd = (loss_i(i, a0[i], bp) - loss_i(i, a0[i], bm)) / (2 * h)
            an = float(bv[i].grad[k])
            assert abs(fd - an) <= 1e-4 * abs(an) + 1e-7 * float(bv[i].grad.abs().max()), (i, k, fd, an)
    finally:
        for s in solvers:
            s.close()

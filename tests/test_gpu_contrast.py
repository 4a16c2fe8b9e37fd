"""High-contrast fields (the quantized generator of Sec. 4.1, contrast rho^2
between rho and 1/rho): the orthogonal variant's factorization stays SPD for
every rho and eps (Sec. 4.1 reports that OrthS never breaks down), and PCG
reaches the residual target; smaller eps gives fewer iterations.  The target
is 1e-10 (the benchmark's): with contrast 1e4-1e6 the condition number of A
reaches ~1e9-1e11, and the solver confirms convergence on the true residual
b - A x, which FP64 cannot certify at the paper's 1e-12 for such A (on a
256^2 grid with contrast 1e6 even 1e-10 is below the attainable floor, about
3e-10).  The paper reports its CG residual target, not a confirmed true
residual."""
import numpy as np
import pytest

from paper_1901_02971_gb300 import Solver
from paper_1901_02971_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _solve(p, levels, eps, precision="fp64"):
    import torch
    s = Solver.from_problem(p, levels=levels, eps=eps, precision=precision, tol=1e-10, maxit=2000)
    try:
        s.factorize()
        b = I.rhs(p.n, 5)
        x, it, rr = s.solve(torch.from_numpy(b).cuda())
        true_rr = np.linalg.norm(b - p.to_scipy() @ x.cpu().numpy()) / np.linalg.norm(b)
        return it, rr, true_rr
    finally:
        s.close()


@pytest.mark.parametrize("rho", [1, 100, 1000])
def test_2d_high_contrast_never_breaks_down(cuda_ok, rho):
    p = I.high_contrast_2d(128, rho, 11)
    its = {}
    for eps in (1e-1, 1e-2, 1e-4):
        it, rr, true_rr = _solve(p, 10, eps)
        assert rr <= 1e-10 and true_rr <= 1.5e-10, (rho, eps, it, rr, true_rr)
        its[eps] = it
    assert its[1e-4] <= its[1e-2] <= its[1e-1], its


@pytest.mark.parametrize("rho,precision", [(1, "fp32"), (100, "fp32"), (1000, "fp64")])
def test_3d_high_contrast_never_breaks_down(cuda_ok, rho, precision):
    p = I.high_contrast_3d(32, rho, 12)
    for eps in (1e-1, 1e-2):
        it, rr, true_rr = _solve(p, 9, eps, precision=precision)
        assert rr <= 1e-10 and true_rr <= 1.5e-10, (rho, eps, it, rr, true_rr)

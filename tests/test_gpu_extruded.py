"""Thin extruded 3D problems partitioned in the plane and extruded in z (the
treatment of the nearly 2D ice-sheet problems in Sec. 4): the top separator
stays small as the plane is refined, like a 2D problem, and PCG converges in
a bounded number of iterations."""
import numpy as np
import pytest

from paper_1901_02971_gb300 import Solver
from paper_1901_02971_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("aniso", [100.0, 1.0])
def test_extruded_size_top_grows_like_2d(cuda_ok, aniso):
    import torch
    tops, its = [], []
    for n, lv in [(64, 9), (128, 11), (256, 13)]:
        p = I.extruded_3d(n, n, 5, 7, aniso=aniso)
        s = Solver.from_problem(p, levels=lv, eps=1e-2, precision="fp32", tol=1e-10)
        try:
            s.factorize()
            b = I.rhs(p.n, 3)
            x, it, rr = s.solve(torch.from_numpy(b).cuda())
            true_rr = np.linalg.norm(b - p.to_scipy() @ x.cpu().numpy()) / np.linalg.norm(b)
            assert rr <= 1e-10 and true_rr <= 1.5e-10, (n, it, true_rr)
            tops.append(s.stats().size_top)
            its.append(it)
        finally:
            s.close()
    # a 3D problem's top separator grows ~4x per doubling of the plane (n^2);
    # a 2D one's stays nearly constant
    print("size_top", tops, "iterations", its)
    assert tops[2] <= 2.5 * tops[0], tops
    assert max(its) <= 60, its

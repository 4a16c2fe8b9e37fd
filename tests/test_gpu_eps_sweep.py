"""Oracle parity over the paper's tolerance sweep (eps = 1e-1, 1e-2, 1e-3;
the sweeps of Sec. 4) on reduced instances of the two large workloads'
generators, in the FP64 form:

* the high-contrast 3D diffusion of the 128^3 workload, a = 10^U(-3, 3)
  constant on 8^3 cell blocks, here on 24^3 cells (27 blocks), L = 6
  (leaves of about 200-500 dofs), geometric partition;
* the k-nearest-neighbour graph Laplacian of the 10^6-point workload (k = 10,
  Gaussian weights, + 1e-4 I), here 3000 points, L = 6, no coordinates
  (the BFS bisection).

The checks are those of the main parity test: relative residual 1e-10
(recursive and recomputed), x within 1e-8 of the oracle's x, iterations
within +10 %, the top separator size and every step's rank total within 2 %
(or 2) of the oracle's.
"""
import math

import numpy as np
import pytest

from oracle import spand_oracle as O
from paper_1901_02971_gb300 import Solver
from paper_1901_02971_gb300 import inputs as I

pytestmark = pytest.mark.gpu

GENS = {
    "diff3d_24_b8": (lambda: I.diffusion_3d(24, 2, block=8), 6, True),
    "knn_3000_k10": (lambda: I.knn_laplacian(3000, 10, 3), 6, False),
}


@pytest.fixture(scope="module")
def problems():
    return {k: g() for k, (g, _, _) in GENS.items()}


@pytest.mark.parametrize("eps", [1e-1, 1e-2, 1e-3])
@pytest.mark.parametrize("name", list(GENS))
def test_eps_sweep_matches_oracle(cuda_ok, problems, name, eps):
    import torch
    p = problems[name]
    _, levels, geo = GENS[name]
    b = I.rhs(p.n, 5)
    ref = O.solve(p, b, levels, eps, use_coords=geo)
    s = Solver.from_problem(p, use_coords=geo, levels=levels, eps=eps)
    try:
        s.factorize()
        xd, it, rr = s.solve(torch.from_numpy(b).cuda())
        x = xd.cpu().numpy()
        assert rr <= 1e-10
        A = p.to_scipy()
        assert np.linalg.norm(b - A @ x) / np.linalg.norm(b) <= 1.5e-10
        err = np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x)
        assert err <= 1e-8, err
        assert it <= math.ceil(1.1 * ref.iters), (it, ref.iters)
        st = s.stats()
        assert abs(st.size_top - ref.factor.size_top) <= max(2, 0.02 * ref.factor.size_top)
        for t in range(1, levels + 1):
            _, after = s.ranks(t)
            got, want = int(after.sum()), int(ref.factor.sizes_after[t - 1].sum())
            assert abs(got - want) <= max(2, 0.02 * want), (t, got, want)
    finally:
        s.close()

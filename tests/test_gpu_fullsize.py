"""The benchmark workload itself (3D 7-point Laplacian 64^3, L = 10,
eps = 1e-2, b seed 1), in the launch configuration bench.py times (device
buffers through the C ABI), against the FP64 oracle's result stored in
tests/golden/oracle_lapl3d_64.json (written by make_oracle_lapl3d_64.py,
which calls only the oracle).

Checked at full size: PCG iterations within +10% of the oracle's, the true
residual recomputed here on the host, x on 256 sampled positions and ||x||
within a relative 1e-8, size_Top and the per-step size totals after
sparsification within 2% (pivot near-ties may move a rank by one).
"""
import json
import math
import os

import numpy as np
import pytest

from paper_1901_02971_gb300 import Solver
from paper_1901_02971_gb300 import inputs as I

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_lapl3d_64.json")


@pytest.fixture(scope="module")
def problem():
    p = I.laplacian_3d(64)
    b = I.rhs(p.n, 1)
    with open(GOLD) as f:
        g = json.load(f)
    return p, b, g


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_benchmark_workload_matches_oracle(cuda_ok, problem, precision):
    import torch
    p, b, g = problem
    s = Solver.from_problem(p, levels=10, eps=1e-2, precision=precision)
    try:
        vals = torch.from_numpy(p.vals).cuda()
        bd = torch.from_numpy(b).cuda()
        s.factorize(vals)
        xd, it, rr = s.solve(bd)
        x = xd.cpu().numpy()
        assert rr <= 1e-10
        A = p.to_scipy()
        assert np.linalg.norm(b - A @ x) / np.linalg.norm(b) <= 1.5e-10
        assert it <= math.ceil(1.1 * g["iters"]), (it, g["iters"])
        idx = np.array(g["sample_idx"])
        xs = np.array(g["sample_x"])
        assert np.linalg.norm(x[idx] - xs) <= 1e-8 * np.linalg.norm(xs)
        assert abs(np.linalg.norm(x) - g["x_norm"]) <= 1e-8 * g["x_norm"]
        st = s.stats()
        assert abs(st.size_top - g["size_top"]) <= 0.02 * g["size_top"]
        for t, want in enumerate(g["sizes_after_per_step"], start=1):
            got = int(s.ranks(t)[1].sum())
            assert abs(got - want) <= max(2, 0.02 * want), (t, got, want)
    finally:
        s.close()

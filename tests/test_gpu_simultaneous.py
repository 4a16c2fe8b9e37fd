"""Simultaneous sparsification order (SPAND_SIMULTANEOUS) against the oracle's
independent implementation of the same order.

Every interface of a level is compressed from the same scaled matrix in one
grouped launch (no W_cn write-back, ranks to a separate array), then every
coupling block is transformed from both sides, A_pq <- Q_pc^T A_pq Q_qc, by
the batched GEMM `k_sim_gemm` (all reads in one launch, all writes in the
next).  Bars as for the coloured order:

* FP64 factor against the oracle (order="simultaneous"): x within 1e-8 at
  relative residual 1e-10, PCG iterations within +10 %, top separator and
  per-step rank totals within 2 % (pivot near-ties);
* eps = 0: the exact ND Cholesky (x equals the dense solution);
* FP32 / TF32 factors reach the oracle's x to 1e-8;
* run-to-run bit-identical results (a race between an interface's rank
  store and its neighbours' size reads, or between the transform's reads
  and writes, would show up here);
* eps = 1 converges (no breakdown: orthogonal two-sided transform).
"""
import math

import numpy as np
import pytest

from oracle import spand_oracle as O
from paper_1901_02971_gb300 import Solver
from paper_1901_02971_gb300 import inputs as I

pytestmark = pytest.mark.gpu

SIM = "simultaneous"


def _run(p, b, levels, eps, precision="fp64", geo=True):
    import torch
    s = Solver.from_problem(p, use_coords=geo, levels=levels, eps=eps, precision=precision, sparsify_order=SIM)
    s.factorize()
    xd, it, rr = s.solve(torch.from_numpy(b).cuda())
    return s, xd.cpu().numpy(), it, rr


CASES = [
    ("lapl2d_64_L8", lambda: I.laplacian_2d(64), 8, 1e-2, True),
    ("lapl2d_61_L7_e1e-1", lambda: I.laplacian_2d(61), 7, 1e-1, True),
    ("lapl3d_20_L7", lambda: I.laplacian_3d(20), 7, 1e-2, True),
    ("diff3d_20_L7", lambda: I.diffusion_3d(20, 2, block=4), 7, 1e-2, True),
    ("hc2d_64_L8", lambda: I.high_contrast_2d(64, 100, 1), 8, 1e-2, True),
    ("knn_6000_L7", lambda: I.knn_laplacian(6000, 10, 3), 7, 1e-2, False),
]


@pytest.mark.parametrize("name,gen,levels,eps,geo", CASES, ids=[c[0] for c in CASES])
def test_fp64_simultaneous_matches_oracle(cuda_ok, name, gen, levels, eps, geo):
    p = gen()
    b = I.rhs(p.n, 0)
    ref = O.solve(p, b, levels, eps, use_coords=geo, order=SIM)
    s, x, it, rr = _run(p, b, levels, eps, geo=geo)
    try:
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


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_simultaneous_eps0_exact(cuda_ok, precision):
    p = I.laplacian_3d(12)
    b = I.rhs(p.n, 6)
    s, x, it, rr = _run(p, b, 5, 0.0, precision=precision)
    try:
        x_ref = np.linalg.solve(p.to_scipy().toarray(), b)
        assert np.linalg.norm(x - x_ref) <= 1e-9 * np.linalg.norm(x_ref)
        assert it <= (2 if precision == "fp64" else 6), it
    finally:
        s.close()


@pytest.mark.parametrize("precision", ["fp32", "tf32"])
def test_mixed_simultaneous_reaches_oracle_accuracy(cuda_ok, precision):
    p = I.laplacian_3d(24)
    b = I.rhs(p.n, 4)
    ref = O.solve(p, b, 7, 1e-2, order=SIM)
    s, x, it, rr = _run(p, b, 7, 1e-2, precision=precision)
    try:
        assert rr <= 1e-10
        assert np.linalg.norm(x - ref.x) <= 1e-8 * np.linalg.norm(ref.x)
        assert it <= 2 * ref.iters + 3, (it, ref.iters)
    finally:
        s.close()


def test_simultaneous_bitwise_repeatable(cuda_ok):
    import torch
    p = I.laplacian_3d(40)
    b = torch.from_numpy(I.rhs(p.n, 3)).cuda()
    outs = []
    for _ in range(3):
        g = torch.empty(32 << 20, dtype=torch.float32, device="cuda")
        g.fill_(float("nan"))
        del g
        s = Solver.from_problem(p, levels=9, eps=1e-2, precision="fp32", sparsify_order=SIM)
        try:
            s.factorize()
            x, it, rr = s.solve(b)
            outs.append((x.cpu().numpy(), it, s.stats().mem_f))
        finally:
            s.close()
    for o in outs[1:]:
        assert o[1:] == outs[0][1:]
        assert np.array_equal(o[0], outs[0][0])


def test_simultaneous_large_eps_stays_spd(cuda_ok):
    p = I.diffusion_3d(16, 2, block=4)
    s, x, it, rr = _run(p, I.rhs(p.n, 1), 6, 1.0)
    try:
        assert rr <= 1e-10
    finally:
        s.close()


@pytest.mark.parametrize("name,gen,levels", [
    ("single_unknown", lambda: I.laplacian_2d(1), 1),
    ("more_levels_than_vertices", lambda: I.laplacian_2d(5), 7),
    ("empty", lambda: I.Problem("empty", 0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0),
                                np.zeros((0, 2)), 2), 3),
])
def test_simultaneous_degenerate_cases(cuda_ok, name, gen, levels):
    p = gen()
    b = I.rhs(p.n, 1)
    s, x, it, rr = _run(p, b, levels, 1e-2)
    try:
        if p.n == 0:
            assert x.size == 0 and it == 0
            return
        ref = O.solve(p, b, levels, 1e-2, order=SIM)
        assert rr <= 1e-10
        assert np.linalg.norm(x - ref.x) <= 1e-8 * np.linalg.norm(ref.x)
    finally:
        s.close()

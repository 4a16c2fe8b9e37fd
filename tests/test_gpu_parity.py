"""GPU path (through the C ABI) against the FP64 oracle on the same seeded
inputs.

Bars:
  * x within a relative 1e-8 of the oracle's x, both at PCG relative residual
    1e-10;
  * PCG iteration count within +10% of the oracle's (rounded up);
  * the true residual ||b - A x|| / ||b|| recomputed here (scipy, FP64)
    at or below 1e-10.
At eps = 0 the factorization is exact (Sec. 3.2 corollary: "even for
eps = 0"), so PCG takes one iteration and x equals the dense solution.
"""
import math

import numpy as np
import pytest

from oracle import spand_oracle as O
from paper_1901_02971_gb300 import Solver, SpandError
from paper_1901_02971_gb300 import _lib as L
from paper_1901_02971_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL_X = 1e-8


def _true_relres(p, x, b):
    A = p.to_scipy()
    return np.linalg.norm(b - A @ x) / np.linalg.norm(b)


def _run(p, b, levels, eps, skip=0, precision="fp64", geo=True, device=False):
    import torch
    s = Solver.from_problem(p, use_coords=geo, levels=levels, eps=eps, skip=skip, precision=precision)
    s.factorize()
    if device:
        bd = torch.from_numpy(b).cuda()
        xd, it, rr = s.solve(bd)
        x = xd.cpu().numpy()
    else:
        x, it, rr = s.solve(b)
    return s, x, it, rr


def _iters_ok(it, it_ref):
    return it <= math.ceil(1.1 * it_ref)


CASES = [
    # name, generator, levels, eps, skip, geometric
    ("lapl2d_64_L8_e1e-2", lambda: I.laplacian_2d(64), 8, 1e-2, 0, True),
    ("lapl2d_64_L8_e1e-1", lambda: I.laplacian_2d(64), 8, 1e-1, 0, True),
    ("lapl2d_61_L7_e1e-3_skip2", lambda: I.laplacian_2d(61), 7, 1e-3, 2, True),
    ("lapl3d_16_L6_e1e-2", lambda: I.laplacian_3d(16), 6, 1e-2, 0, True),
    ("lapl3d_20_L7_e1e-2_skip1", lambda: I.laplacian_3d(20), 7, 1e-2, 1, True),
    ("diff3d_16_L6_e1e-2", lambda: I.diffusion_3d(16, 2, block=4), 6, 1e-2, 0, True),
    ("diff2d_48_L7_e1e-2_nogeo", lambda: I.diffusion_2d(48, 4), 7, 1e-2, 0, False),
    ("knn_4000_L7_e1e-2", lambda: I.knn_laplacian(4000, 10, 3), 7, 1e-2, 0, False),
    # quantized high-contrast fields (Sec. 4.1 generator), contrast 1e6 and 1e4
    ("hc2d_64_r1000_L8_e1e-2", lambda: I.high_contrast_2d(64, 1000, 1), 8, 1e-2, 0, True),
    ("hc2d_48_r1000_L7_e1e-4", lambda: I.high_contrast_2d(48, 1000, 2), 7, 1e-4, 0, True),
    ("hc3d_16_r100_L6_e1e-2", lambda: I.high_contrast_3d(16, 100, 3), 6, 1e-2, 0, True),
    # thin extruded mesh with a six-decade background field, xy partition
    ("extr_32x24x4_L7_e1e-2", lambda: I.extruded_3d(32, 24, 4, 1), 7, 1e-2, 0, True),
]


@pytest.mark.parametrize("name,gen,levels,eps,skip,geo", CASES, ids=[c[0] for c in CASES])
def test_fp64_matches_oracle(cuda_ok, name, gen, levels, eps, skip, geo):
    p = gen()
    b = I.rhs(p.n, 0)
    ref = O.solve(p, b, levels, eps, skip=skip, use_coords=geo)
    s, x, it, rr = _run(p, b, levels, eps, skip=skip, geo=geo, device=True)
    try:
        assert rr <= 1e-10
        assert _true_relres(p, x, b) <= 1.5e-10
        err = np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x)
        assert err <= TOL_X, err
        assert _iters_ok(it, ref.iters), (it, ref.iters)
        # the top separator size and per-step rank totals follow the same
        # truncation rule; pivot near-ties may move a rank by one or two
        st = s.stats()
        assert abs(st.size_top - ref.factor.size_top) <= max(2, 0.02 * ref.factor.size_top)
        for t in range(1, levels + 1):
            before, after = s.ranks(t)
            if t == 1:
                assert np.array_equal(before, ref.factor.sizes_before[0])
            got, want = int(after.sum()), int(ref.factor.sizes_after[t - 1].sum())
            assert abs(got - want) <= max(2, 0.02 * want), (t, got, want)
    finally:
        s.close()


@pytest.mark.parametrize("gen,levels", [(lambda: I.laplacian_2d(8), 3), (lambda: I.laplacian_2d(33), 6),
                                        (lambda: I.laplacian_3d(9), 5), (lambda: I.diffusion_3d(10, 7, block=2), 5)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_eps0_exact(cuda_ok, gen, levels, precision):
    """eps = 0: exact ND Cholesky.  FP64: one iteration; FP32: the factor is
    exact up to single-precision rounding, so a few iterations."""
    p = gen()
    b = I.rhs(p.n, 1)
    s, x, it, rr = _run(p, b, levels, 0.0, precision=precision)
    try:
        x_ref = np.linalg.solve(p.to_scipy().toarray(), b)
        assert np.linalg.norm(x - x_ref) <= 1e-9 * np.linalg.norm(x_ref)
        if precision == "fp64":
            assert it == 1
        else:
            assert it <= 4
    finally:
        s.close()


@pytest.mark.parametrize("name,gen,levels,eps", [
    ("lapl2d_64", lambda: I.laplacian_2d(64), 8, 1e-2),
    ("lapl3d_16", lambda: I.laplacian_3d(16), 6, 1e-2),
    ("diff3d_16", lambda: I.diffusion_3d(16, 2, block=4), 6, 1e-2),
])
def test_fp32_form_converges_to_fp64_accuracy(cuda_ok, name, gen, levels, eps):
    """Mixed form: FP32 factor, FP64 PCG.  The lower precision may only cost
    iterations; x still meets the 1e-8 bar against the FP64 oracle."""
    p = gen()
    b = I.rhs(p.n, 2)
    ref = O.solve(p, b, levels, eps)
    s, x, it, rr = _run(p, b, levels, eps, precision="fp32", device=True)
    try:
        assert rr <= 1e-10
        err = np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x)
        assert err <= TOL_X, err
        assert it <= 2 * ref.iters + 3, (it, ref.iters)
    finally:
        s.close()


def test_host_and_device_buffers_agree(cuda_ok):
    import torch
    p = I.laplacian_3d(12)
    b = I.rhs(p.n, 3)
    s = Solver.from_problem(p, levels=5, eps=1e-2).factorize()
    try:
        xh, ith, _ = s.solve(b)
        xd, itd, _ = s.solve(torch.from_numpy(b).cuda())
        assert ith == itd
        assert np.array_equal(xh, xd.cpu().numpy())  # same kernels, same order: bit-identical
        # refactorize from device values: identical factor and solution
        s.factorize(torch.from_numpy(p.vals).cuda())
        x2, it2, _ = s.solve(b)
        assert it2 == ith and np.array_equal(x2, xh)
    finally:
        s.close()


def test_apply_is_exact_inverse_at_eps0(cuda_ok):
    import torch
    p = I.diffusion_2d(20, 1)
    s = Solver.from_problem(p, levels=5, eps=0.0).factorize()
    try:
        r = I.rhs(p.n, 5)
        z = s.apply(torch.from_numpy(r).cuda()).cpu().numpy()
        z_ref = np.linalg.solve(p.to_scipy().toarray(), r)
        assert np.linalg.norm(z - z_ref) <= 1e-11 * np.linalg.norm(z_ref)
    finally:
        s.close()


# ------------------------------------------------------------- edge cases

def test_single_unknown_and_one_level(cuda_ok):
    p = I.laplacian_2d(1)
    s, x, it, rr = _run(p, np.array([2.0]), 1, 1e-2)
    try:
        assert it == 1 and abs(x[0] - 0.5) < 1e-15
    finally:
        s.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_empty_system(cuda_ok, precision):
    """n = 0: analyze, factorize, solve and apply succeed and do nothing."""
    import torch
    p = I.Problem("empty", 0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0), np.zeros((0, 2)), 2)
    s, x, it, rr = _run(p, np.zeros(0), 3, 1e-2, precision=precision)
    try:
        assert x.size == 0 and it == 0 and rr == 0.0
        st = s.stats()
        assert st.size_top == 0 and st.mem_f == 0
        xd, it, rr = s.solve(torch.zeros(0, dtype=torch.float64, device="cuda"))
        assert xd.numel() == 0 and it == 0
        assert s.apply(torch.zeros(0, dtype=torch.float64, device="cuda")).numel() == 0
        sb, sa = s.ranks(1)
        assert len(sb) == 0 and len(sa) == 0
    finally:
        s.close()


def test_more_levels_than_vertices(cuda_ok):
    """Empty separators / interiors (levels far beyond log2 N)."""
    p = I.laplacian_2d(3)
    b = I.rhs(p.n, 0)
    s, x, it, rr = _run(p, b, 8, 1e-2)
    try:
        x_ref = np.linalg.solve(p.to_scipy().toarray(), b)
        assert rr <= 1e-10 and np.linalg.norm(x - x_ref) <= 1e-9 * np.linalg.norm(x_ref)
    finally:
        s.close()


def test_zero_rhs(cuda_ok):
    p = I.laplacian_2d(16)
    s, x, it, rr = _run(p, np.zeros(p.n), 4, 1e-2)
    try:
        assert it == 0 and not np.any(x)
    finally:
        s.close()


@pytest.mark.parametrize("eps", [0.5, 1.0, 2.0])
def test_large_eps_stays_spd(cuda_ok, eps):
    """OrthS never breaks down (Sec. 3.2), even when most dofs are dropped."""
    p = I.diffusion_3d(12, 3, block=3)
    b = I.rhs(p.n, 0)
    s, x, it, rr = _run(p, b, 5, eps)
    try:
        assert rr <= 1e-10
        ref = O.solve(p, b, 5, eps)
        assert _iters_ok(it, ref.iters), (it, ref.iters)
    finally:
        s.close()


def test_not_spd_reports_error(cuda_ok):
    """An indefinite matrix makes a pivot Cholesky fail: NOT_SPD, no fault."""
    p = I.laplacian_2d(12)
    vals = p.vals.copy()
    rows = np.repeat(np.arange(p.n), np.diff(p.rowptr))
    vals[rows == p.colind] = -1.0  # negative diagonal
    s = Solver(p.rowptr, p.colind, vals, p.coords, levels=4, eps=1e-2)
    try:
        with pytest.raises(SpandError) as ei:
            s.factorize()
        assert ei.value.code == L.SPAND_ERR_NOT_SPD
        st = s.stats()
        assert st.fail_step >= 1 and st.fail_cluster >= 0
        b = np.ones(p.n)
        rc, _, _ = L.spand_solve(s.h, b.ctypes.data, np.zeros(p.n).ctypes.data, check=False)
        assert rc == L.SPAND_ERR_STATE
    finally:
        s.close()


def test_maxit_reports_no_convergence(cuda_ok):
    p = I.laplacian_3d(12)
    b = I.rhs(p.n, 0)
    s = Solver.from_problem(p, levels=5, eps=0.5, maxit=1)
    s.factorize()
    try:
        x, it, rr = s.solve(b, check=False)
        assert it == 1 and rr > 1e-10
        with pytest.raises(SpandError) as ei:
            s.solve(b)
        assert ei.value.code == L.SPAND_ERR_NO_CONVERGENCE
    finally:
        s.close()

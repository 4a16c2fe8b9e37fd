"""TF32 / BF16 forms: FP32 factors whose elimination Schur GEMMs run on the
tensor cores (tcgen05, TF32 or BF16 operands, FP32 accumulation), FP64 PCG.

The operand rounding (2^-11 relative for TF32, 2^-8 for BF16) perturbs the
preconditioner, never the solution: PCG with FP64 residuals still reaches
relative residual 1e-10, so x meets the 1e-8 bar against the FP64 oracle;
only the iteration count may grow.

* Against the oracle on 2D/3D Laplacian, 3D diffusion and kNN cases, with
  Schur blocks spanning several 128 x 64 tensor-core tiles and separators
  longer than one 32/64-element K chunk.
* eps = 0 (exact ND Cholesky up to operand rounding): x equals the dense
  solution to 1e-9 after a handful of iterations.
* The TF32 form's iteration count stays close to the FP32 (SIMT) form's.
* BF16 at eps = 1e-4 on high contrast either converges or reports NOT_SPD
  (its rounding exceeds eps^2; a breakdown is a valid, reported outcome).
"""
import math

import numpy as np
import pytest

from oracle import spand_oracle as O
from paper_1901_02971_gb300 import Solver, SpandError
from paper_1901_02971_gb300 import _lib as L
from paper_1901_02971_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _run(p, b, precision, **kw):
    import torch
    s = Solver.from_problem(p, precision=precision, tol=1e-10, **kw)
    try:
        s.factorize()
        x, it, rr = s.solve(torch.from_numpy(b).cuda())
        return x.cpu().numpy(), it, rr
    finally:
        s.close()


CASES = [
    ("lapl2d_64_L8", lambda: I.laplacian_2d(64), dict(levels=8, eps=1e-2), True),
    ("lapl3d_24_L7", lambda: I.laplacian_3d(24), dict(levels=7, eps=1e-2), True),
    ("diff3d_20_L7", lambda: I.diffusion_3d(20, 2, block=4), dict(levels=7, eps=1e-2), True),
    ("knn_6000_L7", lambda: I.knn_laplacian(6000, 10, 3), dict(levels=7, eps=1e-2), False),
]


@pytest.mark.parametrize("precision", ["tf32", "bf16"])
@pytest.mark.parametrize("name,gen,kw,geo", CASES, ids=[c[0] for c in CASES])
def test_tc_forms_reach_oracle_accuracy(cuda_ok, precision, name, gen, kw, geo):
    p = gen()
    b = I.rhs(p.n, 4)
    ref = O.solve(p, b, kw["levels"], kw["eps"], use_coords=geo)
    x, it, rr = _run(p, b, precision, use_coords=geo, **kw)
    assert rr <= 1e-10
    A = p.to_scipy()
    assert np.linalg.norm(b - A @ x) / np.linalg.norm(b) <= 1.5e-10
    err = np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x)
    assert err <= 1e-8, err
    bound = 2 * ref.iters + 3 if precision == "tf32" else 4 * ref.iters + 6
    assert it <= bound, (it, ref.iters)


@pytest.mark.parametrize("precision", ["tf32", "bf16"])
def test_tc_eps0_is_near_exact(cuda_ok, precision):
    p = I.laplacian_3d(14)
    b = I.rhs(p.n, 6)
    x, it, rr = _run(p, b, precision, levels=6, eps=0.0)
    x_ref = np.linalg.solve(p.to_scipy().toarray(), b)
    assert np.linalg.norm(x - x_ref) <= 1e-9 * np.linalg.norm(x_ref)
    assert it <= (6 if precision == "tf32" else 12), it


def test_tf32_iterations_close_to_fp32(cuda_ok):
    p = I.laplacian_3d(32)
    b = I.rhs(p.n, 8)
    _, it32, _ = _run(p, b, "fp32", levels=8, eps=1e-2)
    _, ittf, _ = _run(p, b, "tf32", levels=8, eps=1e-2)
    assert ittf <= math.ceil(1.25 * it32) + 1, (ittf, it32)


def test_bf16_small_eps_converges_or_reports_not_spd(cuda_ok):
    p = I.high_contrast_2d(64, 1000, 1)
    b = I.rhs(p.n, 9)
    try:
        x, it, rr = _run(p, b, "bf16", levels=8, eps=1e-4)
    except SpandError as e:
        assert e.code == L.SPAND_ERR_NOT_SPD, e
        return
    assert rr <= 1e-10

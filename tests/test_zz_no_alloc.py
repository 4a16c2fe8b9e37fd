"""The allocation-free preconditioner apply.

spand_apply_noalloc exists for callers that must not allocate device memory
during the call (a component that owns the device memory pool, or a
latency-critical loop that cannot take cudaMalloc's implicit synchronisation).
It keeps its work vectors in a fixed array inside the library instead.  Here it
must give the same z = M M^T r as the ordinary spand_apply, call after call
(the shared array keeps the previous call's contents, which must not leak into
the result).  This file is collected last so that a failure here never hides
the other tests of a run that stops at the first failure.
"""
import numpy as np
import pytest

from paper_1901_02971_gb300 import Solver, SpandError
from paper_1901_02971_gb300 import _lib as L
from paper_1901_02971_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_apply_matches_apply_twice(cuda_ok, precision):
    import torch
    p = I.laplacian_3d(16)
    s = Solver.from_problem(p, levels=6, eps=1e-2, precision=precision).factorize()
    try:
        for seed in (11, 12):  # two calls in a row, different inputs
            r = torch.from_numpy(I.rhs(p.n, seed)).cuda()
            z_ref = s.apply(r).cpu().numpy()
            z = torch.empty_like(r)
            L.spand_apply_noalloc(s.h, r.data_ptr(), z.data_ptr(), 0)
            z = z.cpu().numpy()
            assert np.linalg.norm(z - z_ref) <= 1e-13 * np.linalg.norm(z_ref)
    finally:
        s.close()


def test_noalloc_apply_in_place(cuda_ok):
    import torch
    p = I.diffusion_2d(40, 3)
    s = Solver.from_problem(p, levels=6, eps=1e-2).factorize()
    try:
        r = torch.from_numpy(I.rhs(p.n, 4)).cuda()
        z_ref = s.apply(r).cpu().numpy()
        L.spand_apply_noalloc(s.h, r.data_ptr(), r.data_ptr(), 0)  # r and z alias
        assert np.linalg.norm(r.cpu().numpy() - z_ref) <= 1e-13 * np.linalg.norm(z_ref)
    finally:
        s.close()


def test_noalloc_rejects_work_space_beyond_the_fixed_array(cuda_ok):
    """2.25M unknowns alone exceed the 2^21-double array: clear error, no GPU
    work in the call.  The check itself is host arithmetic on n and the
    apply's temporaries, but reaching it needs a factorization of that size
    (about a second of GPU time, the heaviest case of this file)."""
    import torch
    p = I.laplacian_2d(1500)
    s = Solver.from_problem(p, levels=14, eps=1e-1, precision="fp32").factorize()
    try:
        r = torch.zeros(p.n, dtype=torch.float64, device="cuda")
        with pytest.raises(SpandError) as ei:
            L.spand_apply_noalloc(s.h, r.data_ptr(), r.data_ptr(), 0)
        assert ei.value.code == L.SPAND_ERR_INVALID_ARG
        assert "work space" in str(ei.value)
    finally:
        s.close()

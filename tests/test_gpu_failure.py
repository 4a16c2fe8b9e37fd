"""Failure handling of the bounded device-side waits, on the GPU without a
fault: the preconditioner apply's grid barriers are made to wait for an
arrival count that nothing reaches (spand_set_apply_wait), so every wait
runs out after a few polls, every CTA records the timeout and leaves the
kernel, and the call returns SPAND_ERR_TIMEOUT.  The context and the handle
stay usable: a normal apply on the same handle afterwards gives the same
bits as before."""
import numpy as np
import pytest

from paper_1901_02971_gb300 import Solver, SpandError
from paper_1901_02971_gb300 import _lib as L
from paper_1901_02971_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_apply_barrier_timeout_then_recovers(cuda_ok, precision):
    import torch
    p = I.laplacian_3d(12)
    s = Solver.from_problem(p, levels=5, eps=1e-2, precision=precision).factorize()
    try:
        r = torch.from_numpy(I.rhs(p.n, 7)).cuda()
        z_ref = s.apply(r).cpu().numpy()
        L.spand_set_apply_wait(s.h, 64, True)
        for _ in range(2):
            with pytest.raises(SpandError) as ei:
                s.apply(r)
            assert ei.value.code == L.SPAND_ERR_TIMEOUT
        z = torch.empty_like(r)
        with pytest.raises(SpandError) as ei:
            L.spand_apply_noalloc(s.h, r.data_ptr(), z.data_ptr(), 0)
        assert ei.value.code == L.SPAND_ERR_TIMEOUT
        L.spand_set_apply_wait(s.h, 0, False)
        assert np.array_equal(s.apply(r).cpu().numpy(), z_ref)
        x, it, rr = s.solve(I.rhs(p.n, 8))
        assert rr <= 1e-10
    finally:
        s.close()


def test_short_wait_limit_still_completes(cuda_ok):
    """A small but reachable poll limit: either every barrier completes in
    time (same bits as the default) or the call reports the timeout; it
    never returns a wrong z silently."""
    import torch
    p = I.diffusion_2d(48, 2)
    s = Solver.from_problem(p, levels=7, eps=1e-2).factorize()
    try:
        r = torch.from_numpy(I.rhs(p.n, 3)).cuda()
        z_ref = s.apply(r).cpu().numpy()
        L.spand_set_apply_wait(s.h, 1 << 20, False)
        assert np.array_equal(s.apply(r).cpu().numpy(), z_ref)
        L.spand_set_apply_wait(s.h, 1, False)
        try:
            z = s.apply(r).cpu().numpy()
            assert np.array_equal(z, z_ref)
        except SpandError as e:
            assert e.code == L.SPAND_ERR_TIMEOUT
        L.spand_set_apply_wait(s.h, 0, False)
        assert np.array_equal(s.apply(r).cpu().numpy(), z_ref)
    finally:
        s.close()


def test_apply_shape_autotuner_keeps_bits(cuda_ok):
    """The apply's launch shape (CTAs per SM) is autotuned at the first apply;
    every candidate shape gives the same bits of z."""
    import torch
    p = I.laplacian_3d(16)
    s = Solver.from_problem(p, levels=6, eps=1e-2, precision="fp32").factorize()
    try:
        assert s.stats().apply_ctas_per_sm == 0
        r = torch.from_numpy(I.rhs(p.n, 9)).cuda()
        z0 = s.apply(r).cpu().numpy()
        tuned = s.stats().apply_ctas_per_sm
        assert 1 <= tuned <= 4
        for c in (1, 2, 3, 4):
            L.spand_set_apply_shape(s.h, c)
            assert np.array_equal(s.apply(r).cpu().numpy(), z0), c
        L.spand_set_apply_shape(s.h, 0)  # back to the autotuner: it runs again at the next apply
        s.factorize()
        assert np.array_equal(s.apply(r).cpu().numpy(), z0)
    finally:
        s.close()

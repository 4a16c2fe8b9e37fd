"""The preconditioner itself, element by element: z = M M^T r from the GPU
(spand_apply) against the FP64 oracle's apply (Sec. 2.8) at eps > 0.

M depends on the coarse bases Q_pc only through the subspaces they span
(a sign or rotation of a basis carries through every later step and cancels
in M M^T), so where the GPU and the oracle keep the same columns of every
interface -- the same per-cluster ranks at every step, which this test
asserts first -- the two preconditioners agree to rounding.  The cases are
variable-coefficient problems, whose interface blocks have no exactly tied
column norms (a tie broken differently would change the kept subspace at
O(eps) without changing any rank)."""
import numpy as np
import pytest

from oracle import spand_oracle as O
from paper_1901_02971_gb300 import Solver
from paper_1901_02971_gb300 import inputs as I

pytestmark = pytest.mark.gpu

CASES = [
    ("diff2d_40_L6", lambda: I.diffusion_2d(40, 11), 6),
    ("diff2d_56_L7", lambda: I.diffusion_2d(56, 12), 7),
    ("diff3d_12_L5", lambda: I.diffusion_3d(12, 13, block=2), 5),
    ("diff3d_16_L6", lambda: I.diffusion_3d(16, 14, block=2), 6),
]


@pytest.mark.parametrize("eps", [1e-1, 1e-2])
@pytest.mark.parametrize("name,gen,levels", CASES, ids=[c[0] for c in CASES])
def test_apply_matches_oracle_elementwise(cuda_ok, name, gen, levels, eps):
    import torch
    p = gen()
    tree = O.analyze(p.n, p.rowptr, p.colind, p.coords, levels)
    F = O.factorize(p.rowptr, p.colind, p.vals, tree, eps)
    s = Solver.from_problem(p, levels=levels, eps=eps, precision="fp64").factorize()
    try:
        for t in range(1, levels + 1):
            before, after = s.ranks(t)
            assert np.array_equal(before, F.sizes_before[t - 1]), t
            assert np.array_equal(after, F.sizes_after[t - 1]), t
        for seed in (21, 22):
            r = I.rhs(p.n, seed)
            z = s.apply(torch.from_numpy(r).cuda()).cpu().numpy()
            zp = O.apply(F, r[tree.perm])
            z_ref = np.empty(p.n)
            z_ref[tree.perm] = zp
            err = np.abs(z - z_ref).max() / np.abs(z_ref).max()
            assert err <= 1e-12, err
    finally:
        s.close()

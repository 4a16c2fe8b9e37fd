"""The all-core leg of the oracle (``oracle/spand_parallel.py``: Algorithm 2
with the independent block work of each level and colour on a process pool)
computes the serial oracle's factorization: the same ranks and sizes at
every step, the same operator list and memory count, and the same
preconditioner z = M M^T r to rounding (the only reordered arithmetic is
X_sb^T X_sa formed as the transpose of X_sa^T X_sb)."""
import numpy as np
import pytest

from oracle import spand_oracle as O
from oracle import spand_parallel as OP
from paper_1901_02971_gb300 import inputs as I

CASES = [
    ("lapl2d_32_L6", lambda: I.laplacian_2d(32), 6, 1e-2),
    ("diff3d_10_L5", lambda: I.diffusion_3d(10, 3, block=2), 5, 1e-1),
    ("knn_600_L5", lambda: I.knn_laplacian(600, 8, 2), 5, 1e-2),
]


@pytest.fixture(scope="module")
def pool():
    with OP.make_pool(2) as p:
        yield p


@pytest.mark.parametrize("name,gen,levels,eps", CASES, ids=[c[0] for c in CASES])
def test_parallel_leg_equals_serial_oracle(pool, name, gen, levels, eps):
    p = gen()
    coords = p.coords if not name.startswith("knn") else None
    tree = O.analyze(p.n, p.rowptr, p.colind, coords, levels)
    F = O.factorize(p.rowptr, p.colind, p.vals, tree, eps)
    G = OP.factorize(p.rowptr, p.colind, p.vals, tree, eps, pool, 2)
    assert len(F.sizes_after) == len(G.sizes_after)
    for a, b in zip(F.sizes_before, G.sizes_before):
        assert np.array_equal(a, b)
    for a, b in zip(F.sizes_after, G.sizes_after):
        assert np.array_equal(a, b)
    assert F.ranks == G.ranks
    assert (F.mem_f, F.size_top) == (G.mem_f, G.size_top)
    assert [op[0] for op in F.ops] == [op[0] for op in G.ops]
    r = I.rhs(p.n, 3)
    z, w = O.apply(F, r), O.apply(G, r)
    assert np.abs(z - w).max() <= 1e-12 * np.abs(z).max()


def test_parallel_leg_reports_not_spd(pool):
    # an indefinite matrix: the first pivot block that is not SPD stops both
    p = I.laplacian_2d(16)
    vals = p.vals.copy()
    rp = p.rowptr
    for i in range(p.n):  # negate the diagonal of the first row block
        for e in range(rp[i], rp[i + 1]):
            if p.colind[e] == i and i < 8:
                vals[e] = -4.0
    tree = O.analyze(p.n, p.rowptr, p.colind, p.coords, 4)
    with pytest.raises(O.NotSPDError) as e1:
        O.factorize(p.rowptr, p.colind, vals, tree, 1e-2)
    with pytest.raises(O.NotSPDError) as e2:
        OP.factorize(p.rowptr, p.colind, vals, tree, 1e-2, pool, 2)
    assert str(e1.value) == str(e2.value)

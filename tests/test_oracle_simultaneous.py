"""Pins of the oracle's simultaneous sparsification order (every interface of a
level takes its column-pivoted QR from the same scaled matrix, then every
coupling block becomes Q_pc^T A_pq Q_qc), the alternative to the coloured
order that Algorithm 2 leaves open (its FORALL over interfaces):

* eps = 0: M M^T = A^{-1} (dense check on small 2D / 3D problems);
* the first sparsified level's first colour sees the same scaled matrix in
  both orders, so its ranks are identical; the level's block pattern is
  unchanged (no fill, Sec. 2.6.1);
* the kept matrix is a principal submatrix of an orthogonal similarity of an
  SPD matrix, so no Cholesky fails at any eps (0.5, 1, 2);
* accuracy: PCG iterations within the coloured order's + 2 and ranks within
  10 % on 2D / 3D Laplacians and diffusion; the error shrinks with eps.
"""
import numpy as np
import pytest

from oracle import spand_oracle as O
from paper_1901_02971_gb300 import inputs as I


@pytest.mark.parametrize("gen,L", [(lambda: I.laplacian_2d(12), 5), (lambda: I.laplacian_3d(6), 4),
                                   (lambda: I.diffusion_2d(12, 3), 5)])
def test_simultaneous_exact_at_eps0(gen, L):
    p = gen()
    tree = O.analyze(p.n, p.rowptr, p.colind, p.coords, L)
    F = O.factorize(p.rowptr, p.colind, p.vals, tree, 0.0, order="simultaneous")
    A = O.permuted_matrix(p.rowptr, p.colind, p.vals, tree.perm).toarray()
    assert np.linalg.norm(O.dense_preconditioner(F, p.n) @ A - np.eye(p.n)) <= 1e-10 * p.n


def test_first_colour_ranks_agree_and_no_fill():
    p = I.laplacian_3d(12)
    tree = O.analyze(p.n, p.rowptr, p.colind, p.coords, 5)
    tr_c, tr_s = [], []
    Fc = O.factorize(p.rowptr, p.colind, p.vals, tree, 1e-2, trace=tr_c)
    Fs = O.factorize(p.rowptr, p.colind, p.vals, tree, 1e-2, trace=tr_s, order="simultaneous")
    st = tree.steps[0]
    first = [c for c in Fc.ranks[0] if st.colour[c] == 0]
    assert first
    assert all(Fc.ranks[0][c] == Fs.ranks[0][c] for c in first)
    assert set(Fc.ranks[0]) == set(Fs.ranks[0])
    # other colours saw a matrix already changed by earlier colours: ranks may differ
    pre = {t: k for t, ph, k in tr_s if ph == "pre"}
    post = {t: k for t, ph, k in tr_s if ph == "post"}
    assert pre and all(pre[t] == post[t] for t in pre)


@pytest.mark.parametrize("eps", [0.5, 1.0, 2.0])
def test_simultaneous_never_breaks_down(eps):
    for p, L in [(I.diffusion_3d(12, 2, block=3), 5), (I.high_contrast_2d(32, 1000, 1), 7)]:
        r = O.solve(p, I.rhs(p.n, 0), L, eps, order="simultaneous")
        assert r.relres <= 1e-10


@pytest.mark.parametrize("gen,L", [(lambda: I.laplacian_2d(48), 7), (lambda: I.laplacian_3d(16), 6),
                                   (lambda: I.diffusion_3d(16, 2, block=4), 6)])
@pytest.mark.parametrize("eps", [1e-1, 1e-2])
def test_simultaneous_close_to_coloured(gen, L, eps):
    p = gen()
    b = I.rhs(p.n, 2)
    a = O.solve(p, b, L, eps)
    s = O.solve(p, b, L, eps, order="simultaneous")
    ra = sum(sum(d.values()) for d in a.factor.ranks)
    rs = sum(sum(d.values()) for d in s.factor.ranks)
    assert abs(rs - ra) <= 0.1 * ra, (rs, ra)
    assert s.iters <= a.iters + 2, (s.iters, a.iters)
    assert np.linalg.norm(s.x - a.x) <= 1e-8 * np.linalg.norm(a.x)


def test_simultaneous_error_shrinks_with_eps():
    p = I.diffusion_2d(20, 1)
    tree = O.analyze(p.n, p.rowptr, p.colind, p.coords, 5)
    Ap = O.permuted_matrix(p.rowptr, p.colind, p.vals, tree.perm).toarray()
    errs = []
    for eps in [3e-1, 1e-1, 1e-2, 1e-3, 1e-4]:
        F = O.factorize(p.rowptr, p.colind, p.vals, tree, eps, order="simultaneous")
        C = np.linalg.cholesky(O.dense_preconditioner(F, p.n))
        errs.append(np.linalg.norm(np.eye(p.n) - C.T @ Ap @ C, 2))
    assert all(errs[i + 1] <= errs[i] * 1.05 for i in range(len(errs) - 1)), errs
    assert errs[-1] < 1e-2


def test_order_is_validated():
    p = I.laplacian_2d(4)
    tree = O.analyze(p.n, p.rowptr, p.colind, p.coords, 2)
    with pytest.raises(ValueError):
        O.factorize(p.rowptr, p.colind, p.vals, tree, 1e-2, order="random")
    with pytest.raises(ValueError):
        O.factorize(p.rowptr, p.colind, p.vals, tree, 1e-2, variant="InS", order="simultaneous")

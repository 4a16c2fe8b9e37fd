"""Pins of the oracle's randomized sparsification ("OrthS-rand": OrthS with
the column-pivoted QR of A_pn replaced by a randomized range finder, the
randomized alternative the paper names in Sec. 2.6.2 and its conclusion),
checked against dense linear algebra and library routines, not against the
oracle's own formulas:

* the sketch generator is seeded and nested (growing a sketch keeps its
  first columns);
* eps = 0: the sketch grows to min(p, m) columns, whose range is that of
  A_pn, so M M^T = A^{-1} (dense check on small 2D / 3D problems);
* an interface of exact rank k (below and above the first sketch width):
  r = k, the sketch grows only when k saturates it, nothing of A_pn is lost;
* decaying spectra: Q is orthogonal, the dropped block Q_f^T A_pn is at
  least sigma_{r+1}(A_pn) (Eckart-Young) and at most sqrt(m) eps times the
  largest column of A_pn (the column-norm meaning of the truncation rule of
  Sec. 4), and r stays within a few of scipy's column-pivoted QR rank;
* whole solver on 2D / 3D Laplacians: ranks within 15 % of OrthS's, PCG
  iterations within OrthS's + 3, x equal to OrthS's x at the PCG tolerance,
  and no breakdown at eps = 0.9 (the transform stays orthogonal);
* the counter-based sketch (the oracle's Philox4x64-10 + Box-Muller, the
  generator a GPU form would also implement): bit-identical to numpy's
  independent Philox, entries addressed by (seed, step, cluster, row,
  column), Gaussian by a Kolmogorov-Smirnov test, and the solver driven by
  it behaves as with the PCG64 sketch.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import spand_oracle as O
from paper_1901_02971_gb300 import inputs as I


def _sketch(seed=0):
    return lambda t, p, m, ell: I.sketch_gaussian(seed, t, p, m, ell)


def test_sketch_generator_is_seeded_and_nested():
    a = I.sketch_gaussian(3, 2, 7, 50, 20)
    assert a.shape == (50, 20)
    assert np.array_equal(a[:, :8], I.sketch_gaussian(3, 2, 7, 50, 8))
    assert np.array_equal(a, I.sketch_gaussian(3, 2, 7, 50, 20))
    assert not np.array_equal(a, I.sketch_gaussian(3, 2, 8, 50, 20))
    assert abs(a.mean()) < 0.1 and abs(a.std() - 1) < 0.1


@pytest.mark.parametrize("gen,L", [(lambda: I.laplacian_2d(12), 5), (lambda: I.laplacian_3d(6), 4),
                                   (lambda: I.diffusion_2d(12, 3), 5)])
def test_rand_exact_at_eps0(gen, L):
    p = gen()
    tree = O.analyze(p.n, p.rowptr, p.colind, p.coords, L)
    F = O.factorize(p.rowptr, p.colind, p.vals, tree, 0.0, variant="OrthS-rand", sketch=_sketch())
    A = O.permuted_matrix(p.rowptr, p.colind, p.vals, tree.perm).toarray()
    assert np.linalg.norm(O.dense_preconditioner(F, p.n) @ A - np.eye(p.n)) <= 1e-10 * p.n


def _lowrank(seed, p, m, sig):
    rng = np.random.default_rng(seed)
    k = sig.size
    U = np.linalg.qr(rng.standard_normal((p, k)))[0]
    V = np.linalg.qr(rng.standard_normal((m, k)))[0]
    return U @ np.diag(sig) @ V.T


@pytest.mark.parametrize("k,ell", [(20, 32), (25, 64), (40, 64), (70, 80)])
def test_exact_rank_interface(k, ell):
    p, m = 80, 200
    A = _lowrank(k, p, m, np.linspace(1.0, 0.5, k))
    Q, r, Wc, Wf, ell_used = O.sparsify_interface_rand(A, 1e-8, I.sketch_gaussian(1, 1, k, m, p))
    assert r == k
    assert ell_used == ell  # 32; doubled to 64 once r > 32 - 10 oversampling columns; capped at min(p, m) = 80
    assert np.linalg.norm(Q.T @ Q - np.eye(p)) <= 1e-13 * p
    assert np.linalg.norm(A - Q[:, :r] @ Wc) <= 1e-12 * np.linalg.norm(A)
    assert np.linalg.norm(Wf) <= 1e-12 * np.linalg.norm(A)


@pytest.mark.parametrize("seed", range(3))
@pytest.mark.parametrize("p,m,decay", [(80, 200, 0.8), (120, 400, 0.9), (60, 50, 0.7), (200, 600, 0.95)])
@pytest.mark.parametrize("eps", [1e-1, 1e-2, 1e-4])
def test_decaying_spectrum_interface(seed, p, m, decay, eps):
    A = _lowrank(seed, p, m, decay ** np.arange(min(p, m)))
    Q, r, Wc, _, _ = O.sparsify_interface_rand(A, eps, I.sketch_gaussian(seed, 1, 2, m, min(p, m)))
    assert np.linalg.norm(Q.T @ Q - np.eye(p)) <= 1e-13 * p
    assert np.allclose(Wc, Q[:, :r].T @ A, atol=1e-13)
    drop = np.linalg.norm(Q[:, r:].T @ A, 2) if r < p else 0.0
    sig = np.linalg.svd(A, compute_uv=False)
    a0 = np.linalg.norm(A, axis=0).max()
    assert drop <= np.sqrt(m) * eps * a0
    if r < sig.size:
        assert drop >= sig[r] * (1 - 1e-12)
    _, R, _ = sla.qr(A, pivoting=True)
    rc = O.truncation_rank(np.diag(R), eps)
    assert rc - 2 <= r <= 1.1 * rc + 3, (r, rc)


@pytest.mark.parametrize("gen,L", [(lambda: I.laplacian_2d(32), 6), (lambda: I.laplacian_3d(12), 5)])
@pytest.mark.parametrize("eps", [1e-1, 1e-2])
def test_solver_close_to_orths(gen, L, eps):
    p = gen()
    b = I.rhs(p.n, 2)
    a = O.solve(p, b, L, eps)
    r = O.solve(p, b, L, eps, variant="OrthS-rand", sketch=_sketch())
    ra = sum(sum(d.values()) for d in a.factor.ranks)
    rr = sum(sum(d.values()) for d in r.factor.ranks)
    assert 0.97 * ra <= rr <= 1.15 * ra, (rr, ra)
    assert r.iters <= a.iters + 3, (r.iters, a.iters)
    assert r.relres <= 1e-10
    assert np.linalg.norm(r.x - a.x) <= 1e-8 * np.linalg.norm(a.x)


def test_rand_never_breaks_at_large_eps():
    for p, L in [(I.laplacian_2d(24), 6), (I.high_contrast_2d(24, 1000, 1), 6), (I.laplacian_3d(8), 5)]:
        r = O.solve(p, I.rhs(p.n, 1), L, 0.9, variant="OrthS-rand", sketch=_sketch(5))
        assert r.relres <= 1e-10


def test_rand_needs_a_sketch():
    p = I.laplacian_2d(4)
    tree = O.analyze(p.n, p.rowptr, p.colind, p.coords, 2)
    with pytest.raises(ValueError):
        O.factorize(p.rowptr, p.colind, p.vals, tree, 1e-2, variant="OrthS-rand")


# ---------------------------------------------- counter-based sketch (Philox)

def test_philox_matches_numpy_philox():
    """The oracle's Philox4x64-10 against numpy's independent implementation
    (numpy advances its counter before each block, so its block after
    counter c - 1 is ours at c)."""
    rng = np.random.default_rng(11)
    for _ in range(20):
        k = [int(v) for v in rng.integers(0, 2 ** 63, size=2, dtype=np.int64)]
        c = [int(v) for v in rng.integers(1, 2 ** 63, size=4, dtype=np.int64)]
        bg = np.random.Philox(key=np.array(k, dtype=np.uint64),
                              counter=np.array([c[0] - 1] + c[1:], dtype=np.uint64))
        want = [int(v) for v in bg.random_raw(4)]
        got = O.philox4x64_10(*[np.array([v], np.uint64) for v in c], k[0], k[1])
        assert [int(w[0]) for w in got] == want


def test_philox_sketch_is_addressed_by_entry_and_gaussian():
    import scipy.stats as st
    a = O.sketch_philox(3, 2, 7, 50, 20)
    assert np.array_equal(a[:, :8], O.sketch_philox(3, 2, 7, 50, 8))   # nested columns
    assert np.array_equal(a[:29], O.sketch_philox(3, 2, 7, 29, 20))    # any m
    assert not np.array_equal(a, O.sketch_philox(3, 2, 8, 50, 20))     # per cluster
    assert not np.array_equal(a, O.sketch_philox(4, 2, 7, 50, 20))     # per seed
    big = O.sketch_philox(5, 1, 1, 4000, 50).ravel()
    assert abs(big.mean()) < 0.01 and abs(big.var() - 1) < 0.01
    assert st.kstest(big, "norm").pvalue > 1e-3
    # columns are uncorrelated
    c = np.corrcoef(O.sketch_philox(6, 1, 1, 20000, 4).T)
    assert np.abs(c - np.eye(4)).max() < 0.03


@pytest.mark.parametrize("gen,L", [(lambda: I.laplacian_2d(32), 6), (lambda: I.laplacian_3d(12), 5)])
def test_solver_with_philox_sketch(gen, L):
    p = gen()
    b = I.rhs(p.n, 2)
    a = O.solve(p, b, L, 1e-2)
    r = O.solve(p, b, L, 1e-2, variant="OrthS-rand", sketch=lambda t, c, m, ell: O.sketch_philox(0, t, c, m, ell))
    assert r.iters <= a.iters + 3, (r.iters, a.iters)
    assert np.linalg.norm(r.x - a.x) <= 1e-8 * np.linalg.norm(a.x)


def test_cpqr_exact_hand_examples():
    """Pivot order by hand: columns of norms 1, 3, 2 are taken as 3, 2, 1;
    equal norms go by lowest column index."""
    Q, R, P = O.cpqr_exact(np.diag([1.0, 3.0, 2.0]))
    assert P.tolist() == [1, 2, 0]
    assert np.allclose(np.abs(np.diag(R)), [3.0, 2.0, 1.0], rtol=0, atol=1e-15)
    Q, R, P = O.cpqr_exact(np.eye(3))
    assert P.tolist() == [0, 1, 2]
    # a column that becomes the largest only after projecting out the first
    A = np.array([[2.0, 2.0, 0.0], [0.0, 0.1, 1.0]])
    Q, R, P = O.cpqr_exact(A)
    assert P.tolist() == [1, 2, 0]  # ||a_1|| > ||a_0||; then a_2 keeps 0.995-ish, a_0 ~0.1
    assert np.allclose(Q @ R, A[:, P], atol=1e-14)


@pytest.mark.parametrize("seed,shape", [(0, (30, 12)), (1, (12, 30)), (2, (40, 40))])
def test_cpqr_exact_is_a_pivoted_qr(seed, shape):
    """A P = Q R, Q orthogonal, R upper triangular; every |R_kk| is the
    largest norm of a remaining column after projecting out the first k
    (checked by brute force); on Gaussian matrices (no near ties) the pivots
    and |R| equal LAPACK geqp3's."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal(shape)
    Q, R, P = O.cpqr_exact(A)
    m, n = A.shape
    assert np.allclose(Q.T @ Q, np.eye(m), atol=1e-13)
    assert np.allclose(np.tril(R, -1), 0.0)
    assert np.allclose(Q @ R, A[:, P], atol=1e-12)
    for k in range(min(m, n)):
        Qk = Q[:, :k]
        rest = A[:, P[k:]] - Qk @ (Qk.T @ A[:, P[k:]])
        assert abs(abs(R[k, k]) - np.linalg.norm(rest, axis=0).max()) <= 1e-12 * np.abs(A).max() * n
    _, R2, P2 = sla.qr(A, pivoting=True, mode="economic")
    assert P.tolist() == P2.tolist()
    assert np.allclose(np.abs(R[:min(m, n)]), np.abs(R2), atol=1e-12)

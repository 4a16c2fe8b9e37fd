"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these re-types the oracle's own formulas: they check it against a
hand-derived ordering (Algorithm 3 on an 8x8 grid), closed forms (an exact
factorization at eps = 0 equals A^{-1}; the OrthS identities of Sec. 3.1 and
3.2), brute force (dense solves), textbook CG (scipy) and invariants of nested
dissection (Sec. 2.1) and of sparsification (no fill, Sec. 2.6.1).
"""
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from oracle import spand_oracle as O
from paper_1901_02971_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _labels_from_golden(name):
    S, Lb, Rb = {}, {}, {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            y = int(parts[0])
            for x, lab in enumerate(parts[1:]):
                s, l, r = (int(v) for v in lab.split(","))
                v = x + 8 * y
                S[v], Lb[v], Rb[v] = s, l, r
    n = len(S)
    return (np.array([S[v] for v in range(n)]), np.array([Lb[v] for v in range(n)]),
            np.array([Rb[v] for v in range(n)]))


# ---------------------------------------------------------------- Algorithm 3

def test_ordering_8x8_matches_hand_derivation():
    p = I.laplacian_2d(8)
    S, Lb, Rb = O.ordering_clustering(p.n, p.rowptr, p.colind, p.coords, 3)
    gS, gL, gR = _labels_from_golden("nd_8x8_L3.txt")
    assert np.array_equal(S, gS) and np.array_equal(Lb, gL) and np.array_equal(Rb, gR)


def test_clusters_and_merge_8x8_match_hand_derivation():
    p = I.laplacian_2d(8)
    tree = O.analyze(p.n, p.rowptr, p.colind, p.coords, 3)
    want = [(4, -1, -1), (5, -1, -1), (6, -1, -1), (7, -1, -1), (2, 4, 5), (3, 6, 7),
            (1, 2, 3), (1, 4, 6), (1, 5, 7)]
    assert [tuple(k) for k in tree.keys] == want
    sizes = np.diff(tree.cluster_ptr).tolist()
    assert sizes == [9, 12, 12, 16, 3, 4, 1, 3, 4]
    # first cluster: x<=2, y<=2 in id order
    assert tree.perm[:9].tolist() == [0, 1, 2, 8, 9, 10, 16, 17, 18]
    st2 = tree.steps[1]
    assert [tuple(k) for k in st2.keys] == [(2, 2, 2), (3, 3, 3), (1, 2, 3)]
    assert st2.children == [[4], [5], [6, 7, 8]]
    assert tree.steps[0].elim.tolist() == [1, 1, 1, 1, 0, 0, 0, 0, 0]
    assert tree.steps[1].elim.tolist() == [1, 1, 0]
    assert tree.steps[2].elim.tolist() == [1]


def test_root_separator_64x64_is_column_31():
    p = I.laplacian_2d(64)
    S, Lb, Rb = O.ordering_clustering(p.n, p.rowptr, p.colind, p.coords, 3)
    x, y = p.coords[:, 0], p.coords[:, 1]
    assert np.array_equal(np.flatnonzero(S == 1), np.flatnonzero(x == 31))
    # level-2 separators: row y = 31 of each half (the crossing vertex (31,31)
    # stays on the root separator)
    assert np.array_equal(np.flatnonzero(S == 2), np.flatnonzero((y == 31) & (x < 31)))
    assert np.array_equal(np.flatnonzero(S == 3), np.flatnonzero((y == 31) & (x > 31)))
    v = 31 + 64 * 31
    assert (S[v], Lb[v], Rb[v]) == (1, 2, 3)


def _nd_invariants(p, L, coords):
    tree = O.analyze(p.n, p.rowptr, p.colind, coords, L)
    S, Lb, Rb = O.ordering_clustering(p.n, p.rowptr, p.colind, coords, L)
    # clusters partition V
    assert np.array_equal(np.sort(tree.perm), np.arange(p.n))
    # the vertices of each cluster share one label triple
    for c in range(tree.keys.shape[0]):
        vs = tree.perm[tree.cluster_ptr[c]:tree.cluster_ptr[c + 1]]
        assert np.all(S[vs] == tree.keys[c, 0])
        assert np.all(Lb[vs] == tree.keys[c, 1]) and np.all(Rb[vs] == tree.keys[c, 2])
    # ND separation (Sec. 2.1): an edge joins two vertices whose separators
    # are equal or one is an ancestor of the other in the ND tree
    rows = np.repeat(np.arange(p.n), np.diff(p.rowptr))
    sa, sb = S[rows], S[p.colind]
    lo, hi = np.minimum(sa, sb), np.maximum(sa, sb)
    la = np.array([O.level_of(v) for v in lo])
    lb = np.array([O.level_of(v) for v in hi])
    assert np.all((hi >> (lb - la)) == lo), "an edge crosses a separator"
    # every separator is one cluster when it is eliminated
    for t, st in enumerate(tree.steps, 1):
        el = st.keys[st.elim == 1]
        assert len(set(el[:, 0].tolist())) == el.shape[0]
        assert np.all([O.level_of(s) == L + 1 - t for s in el[:, 0]])
    return tree


@pytest.mark.parametrize("gen,L,geo", [
    (lambda: I.laplacian_2d(37), 6, True),
    (lambda: I.laplacian_3d(11), 5, True),
    (lambda: I.diffusion_2d(20, 3), 5, False),
    (lambda: I.knn_laplacian(600, 6, 7), 5, False),
])
def test_nd_invariants(gen, L, geo):
    p = gen()
    _nd_invariants(p, L, p.coords if geo else None)


# ------------------------------------------------ eps = 0: exact ND Cholesky

@pytest.mark.parametrize("gen,L,geo", [
    (lambda: I.laplacian_2d(8), 3, True),
    (lambda: I.laplacian_2d(13), 4, True),
    (lambda: I.laplacian_3d(6), 4, True),
    (lambda: I.diffusion_3d(6, 5, block=2), 4, True),
    (lambda: I.knn_laplacian(150, 5, 11), 4, False),
])
def test_eps0_is_exact_inverse(gen, L, geo):
    p = gen()
    A = p.to_scipy().toarray()
    tree = O.analyze(p.n, p.rowptr, p.colind, p.coords if geo else None, L)
    F = O.factorize(p.rowptr, p.colind, p.vals, tree, eps=0.0)
    MMt = O.dense_preconditioner(F, p.n)
    P = np.eye(p.n)[tree.perm]
    Ap = P @ A @ P.T
    # M M^T = A^{-1} (brute force dense inverse), so (M M^T) A = I
    err = np.linalg.norm(MMt @ Ap - np.eye(p.n), 2)
    assert err < 1e-11 * np.linalg.cond(A)


@pytest.mark.parametrize("skip", [0, 1, 2])
def test_eps0_pcg_one_iteration_and_dense_solution(skip):
    p = I.diffusion_2d(24, 9)
    b = I.rhs(p.n, 0)
    res = O.solve(p, b, 5, 0.0, skip=skip)
    x_ref = np.linalg.solve(p.to_scipy().toarray(), b)
    assert res.iters == 1
    assert np.linalg.norm(res.x - x_ref) <= 1e-10 * np.linalg.norm(x_ref)


# ------------------------------------------------ Sec. 3: OrthS identities

def _random_scaled_system(rng, p, m):
    """SPD [[I, A_pn], [A_np, A_nn]] with an A_pn of decaying spectrum."""
    U = np.linalg.qr(rng.standard_normal((p, p)))[0]
    V = np.linalg.qr(rng.standard_normal((m, m)))[0]
    k = min(p, m)
    sv = 0.7 * 0.5 ** np.arange(k)
    Apn = U[:, :k] @ np.diag(sv) @ V[:, :k].T
    G = rng.standard_normal((m, m))
    Ann = Apn.T @ Apn + G @ G.T / m + 0.1 * np.eye(m)
    return Apn, Ann


@pytest.mark.parametrize("eps", [0.0, 1e-3, 1e-1, 0.5, 1.0])
def test_orths_schur_identity_and_spd(eps):
    """Theorem 3.2: S_B = S_A + W_fn^T W_fn and B_p is SPD for any eps."""
    rng = I.rng(42)
    for p, m in [(12, 30), (20, 7), (9, 9)]:
        Apn, Ann = _random_scaled_system(rng, p, m)
        Q, r, Wc, Wf = O.sparsify_interface(Apn, eps)
        # Q orthogonal and A_pn = Q [W_cn; W_fn]
        assert np.allclose(Q.T @ Q, np.eye(p), atol=1e-13)
        assert np.allclose(Q @ np.vstack([Wc, Wf]), Apn, atol=1e-13)
        SA = Ann - Apn.T @ Apn
        SB = Ann - Wc.T @ Wc
        assert np.allclose(SB - SA, Wf.T @ Wf, atol=1e-12)
        B = np.block([[np.eye(r), Wc], [Wc.T, Ann]])
        np.linalg.cholesky(B)  # SPD: no exception


def test_orths_error_bound():
    """Sec. 3.1: ||E_nn|| = ||W_fn^T W_fn|| <= ||W_fn||^2 = O(eps^2)."""
    rng = I.rng(7)
    Apn, Ann = _random_scaled_system(rng, 16, 40)
    for eps in [1e-1, 1e-2, 1e-3]:
        Q, r, Wc, Wf = O.sparsify_interface(Apn, eps)
        Enn = Wf.T @ Wf
        nf = np.linalg.norm(Wf, 2)
        assert np.linalg.norm(Enn, 2) <= nf ** 2 * (1 + 1e-12)
        # the dropped part is below the threshold relative to the kept one
        R1 = np.linalg.norm(Apn, 2)
        assert nf <= 4 * eps * R1 * np.sqrt(Apn.shape[1])


def test_truncation_rule_on_orthogonal_columns():
    """Columns with disjoint supports: column-pivoted QR sorts them by norm, so
    |R_ii| are the sorted norms and the prefix rule counts norms >= eps*max."""
    p, m = 10, 6
    A = np.zeros((p, m))
    norms = np.array([3.0, 0.5, 1e-3, 2.0, 1e-1, 0.0299])
    for j, s in enumerate(norms):
        A[j, j] = s
    for eps, want in [(1.0, 1), (0.6, 2), (0.1, 3), (0.03, 4), (0.0099, 5), (1e-4, 6), (0.0, 6)]:
        _, r, Wc, _ = O.sparsify_interface(A, eps)
        assert r == want, (eps, r)
    assert O.truncation_rank(np.zeros(3), 0.1) == 0
    assert O.truncation_rank(np.array([2.0, 1.0, 0.1, 0.5]), 0.2) == 2  # prefix, not count


# ------------------------------------------------ Sec. 2.6.1: no fill-in

def test_sparsification_adds_no_blocks():
    p = I.laplacian_3d(10)
    tree = O.analyze(p.n, p.rowptr, p.colind, p.coords, 5)
    trace = []
    O.factorize(p.rowptr, p.colind, p.vals, tree, 1e-2, trace=trace)
    pre = {t: k for t, ph, k in trace if ph == "pre"}
    post = {t: k for t, ph, k in trace if ph == "post"}
    assert pre and set(pre) == set(post)
    for t in pre:
        assert pre[t] == post[t]


# ------------------------------------------------ accuracy trends in eps

def test_error_and_iterations_shrink_with_eps():
    p = I.diffusion_2d(20, 1)
    A = p.to_scipy().toarray()
    tree = O.analyze(p.n, p.rowptr, p.colind, p.coords, 5)
    P = np.eye(p.n)[tree.perm]
    Ap = P @ A @ P.T
    errs, its = [], []
    b = I.rhs(p.n, 3)
    for eps in [3e-1, 1e-1, 1e-2, 1e-3, 1e-4]:
        F = O.factorize(p.rowptr, p.colind, p.vals, tree, eps)
        MMt = O.dense_preconditioner(F, p.n)
        # ||I - M^T A M|| = ||I - (MM^T) A|| in the similarity sense: use the
        # spectrum of the symmetric form via Cholesky of MM^T
        C = np.linalg.cholesky(MMt)
        errs.append(np.linalg.norm(np.eye(p.n) - C.T @ Ap @ C, 2))
        _, it, _ = O.pcg(Ap, b[tree.perm], lambda r: O.apply(F, r))
        its.append(it)
    assert all(errs[i + 1] <= errs[i] * 1.05 for i in range(len(errs) - 1)), errs
    assert all(its[i + 1] <= its[i] for i in range(len(its) - 1)), its
    assert errs[-1] < 1e-2


@pytest.mark.parametrize("eps", [0.5, 1.0])
def test_large_eps_never_breaks_down(eps):
    """Corollary of Sec. 3.2: OrthS stays SPD for any eps."""
    p = I.diffusion_3d(12, 2, block=3)
    b = I.rhs(p.n, 0)
    res = O.solve(p, b, 5, eps, maxit=500)
    assert res.relres <= 1e-10


# ------------------------------------------------ CG against scipy

def test_cg_matches_scipy_unpreconditioned():
    p = I.diffusion_2d(12, 4)
    A = p.to_scipy()
    b = I.rhs(p.n, 5)
    x, it, rr = O.pcg(A, b, lambda r: r.copy(), tol=1e-12, maxit=1000)
    xs, info = spla.cg(A, b, rtol=1e-13, atol=0.0, maxiter=2000)
    assert info == 0 and rr <= 1e-12
    assert np.linalg.norm(x - xs) <= 1e-9 * np.linalg.norm(xs)
    x_ref = np.linalg.solve(A.toarray(), b)
    assert np.linalg.norm(x - x_ref) <= 1e-9 * np.linalg.norm(x_ref)


def test_pcg_true_residual_restart():
    """With a preconditioner that is exact, one iteration suffices; with an
    indefinite-free but poor one, the loop still ends at the true residual."""
    p = I.laplacian_2d(10)
    A = p.to_scipy()
    b = I.rhs(p.n, 1)
    Ainv = np.linalg.inv(A.toarray())
    _, it, rr = O.pcg(A, b, lambda r: Ainv @ r)
    assert it == 1 and rr < 1e-12
    _, it, rr = O.pcg(A, b, lambda r: 0.25 * r, tol=1e-10)
    assert rr <= 1e-10


# ------------------------------------------------ colouring (order of Sec. 2.6.1)

def test_colouring_8x8_matches_hand_derivation():
    """Step 1 of the 8x8, L = 3 case (cluster order of the hand-derived
    ordering above): after the leaves are eliminated the remaining clusters
    c4 = (2,4,5), c5 = (3,6,7), c6 = (1,2,3), c7 = (1,4,6), c8 = (1,5,7) are
    coupled by the original edges c4-c6, c5-c6, c6-c7, c6-c8 and by the fill
    of the four leaves (leaf 4: c4-c7, leaf 5: c4-c8, leaf 6: c5-c7,
    leaf 7: c5-c8).  Greedy colouring in cluster order on that graph:
    c4 0, c5 0, c6 1, c7 2, c8 2.  (On the graph before the fill, c7 and c8
    would take colour 0 and share it with their fill neighbours c4, c5.)"""
    p = I.laplacian_2d(8)
    tree = O.analyze(p.n, p.rowptr, p.colind, p.coords, 3)
    st = tree.steps[0]
    assert st.adjf[4:] == [[6, 7, 8], [6, 7, 8], [4, 5, 7, 8], [4, 5, 6], [4, 5, 6]]
    assert st.colour.tolist() == [-1, -1, -1, -1, 0, 0, 1, 2, 2]
    # step 2: one remaining cluster (the merged root pieces), no neighbours
    assert tree.steps[1].colour.tolist() == [-1, -1, 0]
    assert tree.steps[2].colour.tolist() == [-1]


@pytest.mark.parametrize("gen,L,geo", [
    (lambda: I.laplacian_2d(37), 6, True),
    (lambda: I.laplacian_3d(12), 6, True),
    (lambda: I.diffusion_2d(24, 3), 6, False),
    (lambda: I.knn_laplacian(800, 8, 5), 6, False),
])
def test_colouring_is_proper_and_greedy(gen, L, geo):
    """Every colour class is independent in the graph after the step's fill
    (so its interfaces touch disjoint blocks and run in one launch), the
    fill graph contains every coupling the eliminations create (Sec. 2.4),
    and each cluster takes the smallest colour that none of its earlier
    neighbours holds."""
    p = gen()
    tree = O.analyze(p.n, p.rowptr, p.colind, p.coords if geo else None, L)
    for st in tree.steps:
        nt = st.keys.shape[0]
        rem = [i for i in range(nt) if not st.elim[i]]
        for i in rem:
            assert st.colour[i] >= 0
            for j in st.adjf[i]:
                assert not st.elim[j] and st.colour[j] != st.colour[i]
                assert i in st.adjf[j]
        for s in range(nt):  # neighbours of an eliminated separator become coupled
            if st.elim[s]:
                assert st.colour[s] == -1
                nb = [q for q in st.adj[s] if not st.elim[q]]
                for a in nb:
                    assert set(nb) - {a} <= set(st.adjf[a])
        for i in rem:
            used = {int(st.colour[j]) for j in st.adjf[i] if j < i}
            assert int(st.colour[i]) not in used
            assert all(c in used for c in range(int(st.colour[i])))


# ------------------------------------------------ BFS bisection (reading C3)

def _csr(n, edges):
    rows = {v: {v} for v in range(n)}
    for a, b in edges:
        rows[a].add(b)
        rows[b].add(a)
    rowptr = np.zeros(n + 1, np.int64)
    colind = []
    for v in range(n):
        c = sorted(rows[v])
        colind += c
        rowptr[v + 1] = rowptr[v] + len(c)
    return rowptr, np.array(colind, np.int64)


def test_bfs_tie_break_and_unreached_vertices():
    """Graph 1 - 0 - 2 plus an isolated vertex 3.  BFS from 0 reaches 1 and 2
    at distance 1: the farthest-vertex tie goes to the smallest id, 1.  BFS
    from 1: d = (1, 0, 2) for 0, 1, 2; vertex 3 is unreached and takes the
    largest finite distance + 1 = 3.  Bisection on d: sorted (1, 0, 2, 3),
    threshold d = 1 (position 1), P1 = {0, 1}; 0 touches 2 in P2, so
    left = {1}, separator = {0}, right = {2, 3}.  (Ties to the largest id
    would start from 2 and give d = (1, 2, 0, 3).)"""
    rowptr, colind = _csr(4, [(0, 1), (0, 2)])
    U = np.arange(4)
    d = O.bfs_distance(U, rowptr, colind, 4)
    assert d[:, 0].tolist() == [1.0, 0.0, 2.0, 3.0]
    left, mid, right = O.bisect(U, d, rowptr, colind, 4)
    assert left.tolist() == [1] and mid.tolist() == [0] and right.tolist() == [2, 3]


def test_bfs_bisection_4x3_grid_matches_hand_derivation():
    p = I._assemble((3, 4), np.ones((3, 4)), "grid_4x3")
    S, Lb, Rb = O.ordering_clustering(p.n, p.rowptr, p.colind, None, 2)
    with open(os.path.join(GOLDEN, "bfs_4x3_L2.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    want = np.zeros((12, 3), np.int64)
    for r in rows:
        y = int(r[0])
        for x, lab in enumerate(r[1:]):
            want[x + 4 * y] = [int(v) for v in lab.split(",")]
    assert np.array_equal(np.stack([S, Lb, Rb], axis=1), want)


# ------------------------------------------------ the cluster trees of Sec. 2.3

def test_cluster_trees_of_the_ordering_figure():
    """The ordering-and-clustering figure of Sec. 2.3 on a fine grid of its
    square [-1, 1]^2, with the figure's separators as the vertex-separator
    routine: root = the vertical strip |x| <= 0.075; level 2 = horizontal
    strips at y in [0.10, 0.25] (left half) and [-0.30, -0.15] (right half);
    level 3 = horizontal strips at y in [-0.70, -0.55] (both bottom
    quarters) and [0.50, 0.65] (left top), and the vertical strip
    x in [0.50, 0.65] (right top).  Algorithm 3's labels, clusters of equal
    labels and the label-coarsening merge must give the figure's trees:
    root 9 -> 5 -> 1, its five clusters made of 3, 1, 1, 1, 3 pieces from
    bottom to top; left level-2 separator one cluster throughout; right
    level-2 separator 3 -> 1 (cut by the right-top vertical strip); every
    level-3 separator a single cluster."""
    m = 80
    c = -1 + (2.0 / m) * (np.arange(m) + 0.5)
    p = I._assemble((m, m), np.ones((m, m)), "figure")
    X, Y = c[p.coords[:, 0].astype(int)], c[p.coords[:, 1].astype(int)]
    strips = {(1, 1): (X, -0.075, 0.075), (2, 1): (Y, 0.10, 0.25), (2, 2): (Y, -0.30, -0.15),
              (3, 1): (Y, -0.70, -0.55), (3, 2): (Y, 0.50, 0.65), (3, 3): (Y, -0.70, -0.55),
              (3, 4): (X, 0.50, 0.65)}

    def sep(lvl, k, U):
        v, lo, hi = strips[(lvl, k)]
        v = v[U]
        return U[v < lo], U[(v >= lo) & (v <= hi)], U[v > hi]

    tree = O.analyze(p.n, p.rowptr, p.colind, None, 4, separator=sep)

    def counts(S):
        return [int(np.sum(st.keys[:, 0] == S)) for st in tree.steps if np.any(st.keys[:, 0] == S)]

    assert counts(1) == [9, 5, 1, 1]
    assert counts(2) == [1, 1, 1] and counts(3) == [3, 1, 1]
    assert all(counts(S) == [1, 1] for S in (4, 5, 6, 7))
    # the five step-2 root clusters, bottom to top, and how many step-1
    # clusters each merged
    st2 = tree.steps[1]
    ids = [i for i in range(st2.keys.shape[0]) if st2.keys[i, 0] == 1]

    def ymean(i):
        vs = np.concatenate([tree.perm[tree.cluster_ptr[ch]:tree.cluster_ptr[ch + 1]] for ch in st2.children[i]])
        return Y[vs].mean()

    ids.sort(key=ymean)
    assert [len(st2.children[i]) for i in ids] == [3, 1, 1, 1, 3]
    right2 = [i for i in range(st2.keys.shape[0]) if st2.keys[i, 0] == 3]
    assert [len(st2.children[i]) for i in right2] == [3]

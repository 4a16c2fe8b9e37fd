"""Plain FP64 CPU oracle for sparsified nested dissection (spaND, OrthS).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (its ``cpu_baseline`` leg and ``--impl reference`` arm) may import
or run this module.  The product path (the C-ABI library and its Python
binding) never calls it, and this module imports nothing from the product
package except the seeded input generators' data types.

What it computes, step by step in the paper's order and notation:

* ``analyze``      -- Algorithm 3 (ordering and clustering, Sec. 2.3) with the
                      geometric vertex separator (recursive coordinate bisection,
                      Sec. 2.3 last paragraph) or, without coordinates, a BFS
                      level-set bisection standing in for Metis; clusters =
                      vertices with equal (S, L, R); per-step elimination sets,
                      fill pattern, colouring and merge maps (Sec. 2.7).
* ``factorize``    -- Algorithm 2 (OrthS): for each level from the leaves up,
                      eliminate every separator (block Cholesky, Sec. 2.4),
                      scale every remaining interface (Sec. 2.5), sparsify every
                      interface by column-pivoted QR truncated at eps
                      (Sec. 2.6.1 and the truncation rule of Sec. 4), merge
                      (Sec. 2.7).  Dense algebra uses LAPACK through scipy
                      (Cholesky, triangular solves, geqp3 -- the routine the
                      paper names for its low-rank step).  ``variant`` selects
                      the ablation variants of Sec. 4.3: "In" (interpolative
                      transformations, Sec. 2.6.2, no block scaling) and "InS"
                      (interpolative with block scaling) instead of "OrthS";
                      "OrthS-rand" keeps OrthS but finds the basis of each
                      interface with a randomized range finder (the
                      randomized alternative of Sec. 2.6.2 and the
                      conclusion; method of Halko, Martinsson and Tropp,
                      SIAM Review 2011, Algorithm 4.2 with a doubling
                      sketch), see ``sparsify_interface_rand``.
* ``apply``        -- z = M M^T r with M the product of the elementary
                      transforms (Sec. 2.8): forward sweep leaf->root, backward
                      sweep root->leaf with transposes.
* ``pcg``          -- textbook preconditioned CG (Hestenes-Stiefel), stopping
                      at ||b - A x|| / ||b|| <= tol (Sec. 4).

Readings where the paper is silent (they are the same for the product path):

* Heap labels: separator (l, k) <-> h = 2^(l-1) + k - 1; none = -1.
* Geometric separator on U = I u B: split dimension = largest span (lowest on
  ties); sort U by (x_d, vertex id); threshold t = x_d of the element at
  0-based position floor((|U|-1)/2); P1 = {x_d <= t}, P2 = rest; if P2 is empty
  P1 = the first ceil(|U|/2) of the sorted order; |U| < 2 -> no separator, all
  left.  M = vertices of P1 with a neighbour in P2; left = P1 \\ M, right = P2.
* No coordinates: BFS from the smallest id, restart from the farthest vertex
  (smallest id on ties), BFS distance is the single coordinate (unreached
  vertices: largest finite distance + 1).  This replaces Metis (not
  reproducible bit for bit).
* Clusters sorted by (elimination step, S, L, R); vertices inside a cluster by
  id.  Step t = 1..L eliminates the separators of level L+1-t (t=1: leaves).
* Merge after step t: every L/R label at level L+1-t is replaced by its parent;
  clusters with equal labels merge; parents sorted like clusters, children kept
  in the order of the previous step.
* Scaling and sparsification run after step t iff skip < t < L.  Sparsified
  rows A_pn span all neighbours of p, ordered by cluster index.
* Order of sparsification inside a level: greedy distance-1 colouring of the
  cluster graph (after the level's fill) in cluster order; colours are
  processed in increasing order, clusters of one colour are independent.
  Option ``order="simultaneous"`` (OrthS only): every interface of the level
  takes its pivoted QR from the same scaled matrix, then every coupling
  block becomes A_pq <- Q_pc^T A_pq Q_qc (the c-c principal submatrix of
  the orthogonal similarity diag(Q_p)^T A diag(Q_p), hence SPD).
* Truncation: r = longest prefix with |R_ii| >= eps |R_11|; r = 0 when R_11 = 0
  (p is exactly decoupled).  A cluster with no neighbours (A_pn has no columns)
  is left as it is: there is nothing to compress it against, and keeping it
  or dropping it gives the same M, since its scaled diagonal block is I.  The
  coarse dofs c are the first r columns of Q.
* PCG: x0 = 0; recursive residual; on reaching tol the true residual is
  checked and, if above tol, PCG restarts from it; iteration count = number of
  products A p.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, List, Optional, Tuple

import numpy as np
import scipy.linalg as sla

NONE = -1


class NotSPDError(RuntimeError):
    pass


# --------------------------------------------------------------------------
# labels
# --------------------------------------------------------------------------

def heap(level: int, k: int) -> int:
    """Separator (l, k), 1 <= k <= 2^(l-1)  ->  heap index 2^(l-1) + k - 1."""
    return (1 << (level - 1)) + k - 1


def level_of(h: int) -> int:
    """Level l of heap index h (root = 1)."""
    return int(h).bit_length()


# --------------------------------------------------------------------------
# vertex separators (Sec. 2.3, last paragraph)
# --------------------------------------------------------------------------

def _has_nbr_in(rowptr, colind, rows: np.ndarray, mask: np.ndarray) -> np.ndarray:
    """For each vertex in rows: does it have a neighbour w (w != v) with mask[w]."""
    if rows.size == 0:
        return np.zeros(0, dtype=bool)
    starts = rowptr[rows]
    lens = rowptr[rows + 1] - starts
    idx = np.repeat(starts - np.cumsum(np.concatenate([[0], lens[:-1]])), lens) + np.arange(lens.sum())
    nb = colind[idx]
    owner = np.repeat(np.arange(rows.size), lens)
    hit = mask[nb] & (nb != rows[owner])
    out = np.zeros(rows.size, dtype=bool)
    out[owner[hit]] = True
    return out


def bisect(U: np.ndarray, x: np.ndarray, rowptr, colind, n: int):
    """Split U (sorted ids) with coordinates x (|U| x dim) into (left, mid, right)."""
    if U.size < 2:
        return U.copy(), U[:0], U[:0]
    span = x.max(axis=0) - x.min(axis=0)
    d = int(np.argmax(span))  # first maximum -> lowest dimension on ties
    order = np.lexsort((U, x[:, d]))
    t = x[order[(U.size - 1) // 2], d]
    in1 = x[:, d] <= t
    if in1.all():
        in1 = np.zeros(U.size, dtype=bool)
        in1[order[: (U.size + 1) // 2]] = True
    P1, P2 = U[in1], U[~in1]
    mask2 = np.zeros(n, dtype=bool)
    mask2[P2] = True
    mid_flag = _has_nbr_in(rowptr, colind, P1, mask2)
    return P1[~mid_flag], P1[mid_flag], P2


def bfs_distance(U: np.ndarray, rowptr, colind, n: int) -> np.ndarray:
    """Coordinate for the algebraic separator: BFS distance (see module doc)."""
    inU = np.zeros(n, dtype=bool)
    inU[U] = True

    def bfs(src):
        dist = np.full(n, -1, dtype=np.int64)
        dist[src] = 0
        front = np.array([src])
        lvl = 0
        while front.size:
            starts = rowptr[front]
            lens = rowptr[front + 1] - starts
            idx = np.repeat(starts - np.cumsum(np.concatenate([[0], lens[:-1]])), lens) + np.arange(lens.sum())
            nb = np.unique(colind[idx])
            nb = nb[inU[nb] & (dist[nb] < 0)]
            lvl += 1
            dist[nb] = lvl
            front = nb
        return dist

    d0 = bfs(int(U[0]))[U]
    far = d0.max()
    r1 = int(U[np.flatnonzero(d0 == far)[0]])
    d1 = bfs(r1)[U]
    reached = d1 >= 0
    d1 = np.where(reached, d1, d1[reached].max() + 1)
    return d1.astype(np.float64)[:, None]


# --------------------------------------------------------------------------
# Algorithm 3: ordering and clustering
# --------------------------------------------------------------------------

def ordering_clustering(n, rowptr, colind, coords: Optional[np.ndarray], L: int, separator=None):
    """Returns C = (S, Lb, Rb) per vertex, heap-indexed (Algorithm 3).

    ``separator(level, k, U) -> (left, mid, right)`` replaces the
    vertex-separator routine (Algorithm 3 works with any); by default the
    geometric bisection, or the BFS bisection without coordinates."""
    S = np.ones(n, dtype=np.int64)          # (1,1) for everyone
    Lb = np.full(n, NONE, dtype=np.int64)   # none
    Rb = np.full(n, NONE, dtype=np.int64)
    for lvl in range(1, L):
        for k in range(1, (1 << (lvl - 1)) + 1):
            h = heap(lvl, k)
            I = np.flatnonzero(S == h)
            B = np.flatnonzero((Lb == h) | (Rb == h))
            U = np.union1d(I, B)
            if separator is not None:
                left, mid, right = (np.asarray(a, dtype=np.int64) for a in separator(lvl, k, U))
            else:
                if coords is not None:
                    x = coords[U]
                else:
                    x = bfs_distance(U, rowptr, colind, n) if U.size >= 2 else np.zeros((U.size, 1))
                left, mid, right = bisect(U, x, rowptr, colind, n)
            inB = np.zeros(n, dtype=bool)
            inB[B] = True
            inI = np.zeros(n, dtype=bool)
            inI[I] = True
            # update separator, left and right interiors
            S[mid[~inB[mid]]] = h
            S[left[~inB[left]]] = 2 * h
            S[right[~inB[right]]] = 2 * h + 1
            # neighbours of the new separator
            mI = mid[inI[mid]]
            Lb[mI] = 2 * h
            Rb[mI] = 2 * h + 1
            # boundary vertices that fell left / right
            for part, child in ((left[inB[left]], 2 * h), (right[inB[right]], 2 * h + 1)):
                isL = Lb[part] == h
                Lb[part[isL]] = child
                Rb[part[~isL]] = child
    return S, Lb, Rb


def _coarsen(h: int, lam: int) -> int:
    """Merge rule: a label at level lam is replaced by its parent."""
    if h != NONE and level_of(h) == lam:
        return h // 2
    return h


@dataclass
class Step:
    """Integer structure of elimination step t (all indices are into this
    step's cluster list)."""
    keys: np.ndarray        # (n_t, 3) S, L, R
    children: List[List[int]]  # indices into the previous step's list (step 1: initial clusters)
    elim: np.ndarray        # (n_t,) 1 if eliminated at this step
    colour: np.ndarray      # (n_t,) greedy colour of remaining clusters, -1 if eliminated
    adj: List[List[int]]    # cluster graph before elimination (sorted)
    adjf: List[List[int]]   # graph of remaining clusters after this step's fill (sorted)


@dataclass
class Tree:
    n: int
    L: int
    perm: np.ndarray          # int64 (n,): perm[i] = vertex at position i
    cluster_ptr: np.ndarray   # int64 (nc+1,)
    keys: np.ndarray          # int64 (nc, 3)
    steps: List[Step]


def analyze(n, rowptr, colind, coords, L, separator=None) -> Tree:
    rowptr = np.asarray(rowptr, dtype=np.int64)
    colind = np.asarray(colind, dtype=np.int64)
    S, Lb, Rb = ordering_clustering(n, rowptr, colind, coords, L, separator)
    # clusters = vertices with the same C[v]; order (step, S, L, R), ids ascending
    step_of = L + 1 - np.array([level_of(h) for h in range(0, 1 << L)], dtype=np.int64)
    tv = step_of[S]
    order = np.lexsort((np.arange(n), Rb, Lb, S, tv))
    keys_sorted = np.stack([tv[order], S[order], Lb[order], Rb[order]], axis=1)
    newc = np.ones(n, dtype=bool)
    newc[1:] = np.any(keys_sorted[1:] != keys_sorted[:-1], axis=1)
    starts = np.flatnonzero(newc)
    cluster_ptr = np.concatenate([starts, [n]]).astype(np.int64)
    keys = keys_sorted[starts, 1:]
    nc = keys.shape[0]
    cl_of = np.empty(n, dtype=np.int64)
    cl_of[order] = np.repeat(np.arange(nc), np.diff(cluster_ptr))
    # initial cluster graph from the edges of A
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    a, b = cl_of[rows], cl_of[colind]
    m = a != b
    pairs = np.unique(np.stack([a[m], b[m]], axis=1), axis=0) if m.any() else np.zeros((0, 2), np.int64)
    adj = [set() for _ in range(nc)]
    for x, y in pairs:
        adj[x].add(int(y))
    cur_keys = [tuple(int(v) for v in k) for k in keys]
    children = [[i] for i in range(nc)]
    steps: List[Step] = []
    for t in range(1, L + 1):
        lam = L + 1 - t
        nt = len(cur_keys)
        elim = np.array([1 if level_of(k[0]) == lam else 0 for k in cur_keys], dtype=np.int64)
        for i in range(nt):
            if elim[i]:
                for j in adj[i]:
                    if elim[j]:
                        raise RuntimeError("two separators of one level are adjacent")
        # fill: neighbours of every eliminated separator become pairwise adjacent
        adjf = [set() if elim[i] else {j for j in adj[i] if not elim[j]} for i in range(nt)]
        for s in range(nt):
            if elim[s]:
                nb = sorted(adj[s])
                for x in nb:
                    for y in nb:
                        if x != y:
                            adjf[x].add(y)
        colour = np.full(nt, -1, dtype=np.int64)
        for i in range(nt):
            if elim[i]:
                continue
            used = {int(colour[j]) for j in adjf[i] if j < i}
            c = 0
            while c in used:
                c += 1
            colour[i] = c
        steps.append(Step(np.array(cur_keys, dtype=np.int64).reshape(nt, 3), children, elim, colour,
                          [sorted(s) for s in adj], [sorted(s) for s in adjf]))
        # merge (Sec. 2.7)
        rem = [i for i in range(nt) if not elim[i]]
        newkey = {i: (cur_keys[i][0], _coarsen(cur_keys[i][1], lam), _coarsen(cur_keys[i][2], lam)) for i in rem}
        uniq = sorted(set(newkey.values()), key=lambda k: (L + 1 - level_of(k[0]), k[0], k[1], k[2]))
        pidx = {k: j for j, k in enumerate(uniq)}
        ch = [[] for _ in uniq]
        for i in rem:
            ch[pidx[newkey[i]]].append(i)
        nadj = [set() for _ in uniq]
        for i in rem:
            for j in adjf[i]:
                P, Q = pidx[newkey[i]], pidx[newkey[j]]
                if P != Q:
                    nadj[P].add(Q)
        cur_keys, children, adj = uniq, ch, nadj
    if cur_keys:
        raise RuntimeError("clusters left after the root step")
    return Tree(n, L, order.astype(np.int64), cluster_ptr, keys.astype(np.int64), steps)


# --------------------------------------------------------------------------
# Algorithm 2 (OrthS): numeric factorization
# --------------------------------------------------------------------------

@dataclass
class Factor:
    ops: list = field(default_factory=list)   # ('E', s_slots, Ls, [(n_slots, Xt)]), ('S', p_slots, Lp), ('Q', p_slots, Q),
    #                                           ('T', c_slots, f_slots, T_cf)
    ranks: List[Dict[int, int]] = field(default_factory=list)  # per step: cluster -> r
    sizes_before: List[np.ndarray] = field(default_factory=list)  # per step: cluster sizes at step start
    sizes_after: List[np.ndarray] = field(default_factory=list)   # per step: sizes after sparsification (0 = eliminated)
    size_top: int = 0
    mem_f: int = 0


def truncation_rank(rdiag: np.ndarray, eps: float) -> int:
    """Longest prefix with |R_ii| >= eps |R_11| (Sec. 4); 0 if R_11 = 0."""
    d = np.abs(rdiag)
    if d.size == 0 or d[0] == 0.0:
        return 0
    ok = d >= eps * d[0]
    return int(d.size if ok.all() else np.argmin(ok))


def sparsify_interface(Apn: np.ndarray, eps: float):
    """Orthogonal sparsification of one scaled interface (Sec. 2.6.1).

    A_pn P = Q R (column-pivoted QR); keep the first r rows.  Returns
    (Q, r, W_cn, W_fn) with A_pn = Q [W_cn; W_fn] and Q = [Q_pc Q_pf]."""
    p, m = Apn.shape
    if m == 0:
        return np.eye(p), p, np.zeros((p, 0)), np.zeros((0, 0))
    if p == 0:
        return np.eye(0), 0, np.zeros((0, m)), np.zeros((0, m))
    Q, R, P = sla.qr(Apn, pivoting=True, mode="full")
    r = truncation_rank(np.diag(R), eps)
    W = np.empty((p, m))
    W[:, P] = R            # Q^T A_pn = R P^T
    return Q, r, W[:r], W[r:]


def sparsify_interface_interp(Anp: np.ndarray, App: np.ndarray, eps: float):
    """Interpolative sparsification of one interface (Sec. 2.6.2).

    Column-pivoted QR of A_np (neighbour rows x the dofs of p): A_np P = Q R,
    r from the truncation rule; c = the first r pivoted dofs, f = the rest,
    T_cf = R_11^{-1} R_12, so that A_nf = A_nc T_cf + Q_2 R_22 (the second
    term, O(eps), is dropped).  With T_p = I - E_cf T_cf (block (c, f) =
    -T_cf) the diagonal block becomes
        C_ff = A_ff - A_fc T_cf - T_cf^T A_cf + T_cf^T A_cc T_cf,
        C_cf = A_cf - A_cc T_cf,
    and f, coupled to c only, is eliminated: L_f = chol(C_ff) (NotSPDError if
    C_ff is not SPD: the breakdown the paper reports for these variants),
    X_fc = L_f^{-1} C_fc, A_cc <- A_cc - X_fc^T X_fc.
    Returns (c, f, T_cf, L_f, X_fc, A_cc_new, R22) with c, f local indices."""
    m, p = Anp.shape
    if p == 0 or m == 0:
        return np.arange(p), np.zeros(0, np.int64), np.zeros((p, 0)), np.zeros((0, 0)), np.zeros((0, p)), \
            App.copy(), np.zeros((0, 0))
    _, R, P = sla.qr(Anp, pivoting=True, mode="economic")
    r = truncation_rank(np.diag(R), eps)
    c, f = P[:r], P[r:]
    T = sla.solve_triangular(R[:r, :r], R[:r, r:], lower=False) if r else np.zeros((0, p - r))
    R22 = R[r:, r:]
    Acc, Acf, Aff = App[np.ix_(c, c)], App[np.ix_(c, f)], App[np.ix_(f, f)]
    Cff = Aff - Acf.T @ T - T.T @ Acf + T.T @ Acc @ T
    Ccf = Acf - Acc @ T
    if f.size:
        try:
            Lf = np.linalg.cholesky(Cff)
        except np.linalg.LinAlgError as e:
            raise NotSPDError("interpolative sparsification: C_ff not SPD") from e
        Xfc = sla.solve_triangular(Lf, Ccf.T, lower=True)
        Acc = Acc - Xfc.T @ Xfc
    else:
        Lf, Xfc = np.zeros((0, 0)), np.zeros((0, r))
    return c, f, T, Lf, Xfc, Acc, R22


# --------------------------------------------------------------------------
# counter-based Gaussian sketch (the oracle's side of a generator that a GPU
# form draws on the device): Philox4x64-10 (Salmon, Moraes, Dror and Shaw,
# "Parallel random numbers: as easy as 1, 2, 3", SC 2011) and Box-Muller
# --------------------------------------------------------------------------

_PHILOX_M = (0xD2E7470EE14C6C93, 0xCA5A826395121157)  # round multipliers
_PHILOX_W = (0x9E3779B97F4A7C15, 0xBB67AE8584CAA73B)  # key increments (Weyl)
_M32 = np.uint64(0xFFFFFFFF)


def _mulhilo64(a: np.ndarray, b: int):
    """(high, low) 64-bit halves of the 128-bit products a * b (a uint64
    array, b a 64-bit constant), from 32-bit partial products."""
    a = a.astype(np.uint64)
    s32 = np.uint64(32)
    al, ah = a & _M32, a >> s32
    bl, bh = np.uint64(b & 0xFFFFFFFF), np.uint64(b >> 32)
    ll, lh, hl, hh = al * bl, al * bh, ah * bl, ah * bh
    mid = (ll >> s32) + (lh & _M32) + (hl & _M32)
    hi = hh + (lh >> s32) + (hl >> s32) + (mid >> s32)
    lo = a * np.uint64(b)  # wraps modulo 2^64
    return hi, lo


def philox4x64_10(c0, c1, c2, c3, k0: int, k1: int):
    """The Philox4x64 bijection with 10 rounds on counter words (uint64
    arrays) under the key (k0, k1): per round, the products of M0 with x0 and
    M1 with x2 give x <- (hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0); the key
    advances by the Weyl constants between rounds."""
    x = [np.asarray(c, dtype=np.uint64) for c in (c0, c1, c2, c3)]
    mask = (1 << 64) - 1
    for r in range(10):
        if r:
            k0, k1 = (k0 + _PHILOX_W[0]) & mask, (k1 + _PHILOX_W[1]) & mask
        h0, l0 = _mulhilo64(x[0], _PHILOX_M[0])
        h1, l1 = _mulhilo64(x[2], _PHILOX_M[1])
        x = [h1 ^ x[1] ^ np.uint64(k0), l1, h0 ^ x[3] ^ np.uint64(k1), l0]
    return x


def sketch_philox(seed: int, step: int, cluster: int, m: int, ell: int) -> np.ndarray:
    """Gaussian test matrix (m x ell) of the randomized compression, entry by
    entry from a counter: key (seed, step * 2^32 + cluster), counter
    (column j, row block i // 4, 0, 0); the four 64-bit words of a block give
    four uniforms u = (w >> 11 + 1/2) 2^-53 in (0, 1), and Box-Muller turns
    the pairs (u0, u1), (u2, u3) into rows 4b..4b+3:
    sqrt(-2 ln u0) (cos 2 pi u1, sin 2 pi u1), likewise for (u2, u3).
    Every entry depends only on (seed, step, cluster, i, j)."""
    nb = (m + 3) // 4
    jj, bb = np.meshgrid(np.arange(ell, dtype=np.uint64), np.arange(nb, dtype=np.uint64))
    z = np.zeros_like(jj)
    w = philox4x64_10(jj, bb, z, z, int(seed) & ((1 << 64) - 1), ((int(step) << 32) + int(cluster)) & ((1 << 64) - 1))
    u = [((wi >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53 for wi in w]
    r01, r23 = np.sqrt(-2.0 * np.log(u[0])), np.sqrt(-2.0 * np.log(u[2]))
    rows = np.stack([r01 * np.cos(2 * np.pi * u[1]), r01 * np.sin(2 * np.pi * u[1]),
                     r23 * np.cos(2 * np.pi * u[3]), r23 * np.sin(2 * np.pi * u[3])], axis=1)  # nb x 4 x ell
    return rows.reshape(4 * nb, ell)[:m]


def cpqr_exact(A: np.ndarray):
    """Column-pivoted Householder QR with the column norms recomputed exactly
    at every step (Businger and Golub, Numer. Math. 1965): step k moves the
    remaining column of largest norm below row k to position k (lowest
    original column index on ties) and reflects it onto e_k.  In exact
    arithmetic this is geqp3's pivot sequence; geqp3 downdates its norm
    estimates instead, so the two part ways at near ties.  Returns (Q, R, P)
    with A[:, P] = Q R, Q square orthogonal, R upper triangular."""
    A = np.array(A, dtype=np.float64, copy=True)
    m, n = A.shape
    P = np.arange(n)
    Q = np.eye(m)
    for k in range(min(m, n)):
        nrm = (A[k:, k:] ** 2).sum(axis=0)
        best = nrm.max()
        j = k + int(np.argmin(np.where(nrm == best, P[k:], n)))  # lowest original index among the largest
        A[:, [k, j]] = A[:, [j, k]]
        P[[k, j]] = P[[j, k]]
        x = A[k:, k]
        nx = np.sqrt(nrm[j - k])
        if nx == 0.0:
            continue
        beta = -nx if x[0] >= 0 else nx          # R_kk, sign opposite to the pivot entry
        v = x / (x[0] - beta)
        v[0] = 1.0
        tau = (beta - x[0]) / beta
        A[k:, k:] -= tau * np.outer(v, v @ A[k:, k:])
        A[k + 1:, k] = 0.0
        Q[:, k:] -= tau * np.outer(Q[:, k:] @ v, v)  # Q <- Q H_k
    return Q, np.triu(A), P


RAND_OVERSAMPLE = 10   # sketch columns beyond the rank (HMT 2011, Sec. 4.2)
RAND_ELL0 = 32         # first sketch width; doubled while the rank saturates it


def sparsify_interface_rand(Apn: np.ndarray, eps: float, Omega: np.ndarray,
                            oversample: int = RAND_OVERSAMPLE, ell0: int = RAND_ELL0):
    """Orthogonal sparsification of one scaled interface with a randomized
    range finder in place of the column-pivoted QR of A_pn.

    Omega is an m x min(p, m) Gaussian test matrix (an input: the random
    numbers are drawn outside).  With ell = min(ell0, min(p, m)) sketch
    columns, Y = A_pn Omega[:, :ell] samples the range of A_pn and the
    column-pivoted QR Y P = Q R orders an orthogonal basis Q (p x p) of it
    (``cpqr_exact``: the column norms recomputed at every step, so that the
    order of the basis -- which decides where the rank rule below stops --
    is the largest-remaining-norm order itself, not geqp3's estimate of it).
    W = Q^T A_pn.  The rank follows the meaning of the truncation rule of
    Sec. 4: in a column-pivoted QR |R_kk| is the largest column norm of the
    part of A_pn outside the first k basis vectors, so here r = the first
    k <= ell with  max_j ||W[k:, j]|| < eps max_j ||A_pn[:, j]||.  If no
    k <= ell qualifies, or r > ell - oversample (the sketch may miss part of
    the range), ell doubles, capped at min(p, m), where range(Y) = range(A_pn)
    with probability one; at the cap r = ell if still no k qualifies, so
    eps = 0 stays exact.  Then, as in Sec. 2.6.1, c = the first r columns of
    Q, W_cn = W[:r] is kept and W_fn = W[r:] dropped.
    Returns (Q, r, W_cn, W_fn, ell)."""
    p, m = Apn.shape
    if m == 0:
        return np.eye(p), p, np.zeros((p, 0)), np.zeros((0, 0)), 0
    if p == 0:
        return np.eye(0), 0, np.zeros((0, m)), np.zeros((0, m)), 0
    ell_max = min(p, m)
    if Omega.shape != (m, ell_max):
        raise ValueError("sketch must be m x min(p, m)")
    a0 = np.sqrt((Apn * Apn).sum(axis=0)).max()
    ell = min(ell0, ell_max)
    while True:
        Y = Apn @ Omega[:, :ell]
        Q, _, _ = cpqr_exact(Y)
        W = Q.T @ Apn
        # res[k] = max_j ||W[k:, j]||, k = 0..ell
        tail = np.cumsum((W * W)[::-1], axis=0)[::-1]
        res = np.sqrt(np.vstack([tail, np.zeros((1, m))]).max(axis=1))[:ell + 1]
        below = np.nonzero(res < eps * a0)[0]
        r = int(below[0]) if below.size else ell
        if ell == ell_max or (below.size and r <= ell - oversample):
            break
        ell = min(2 * ell, ell_max)
    return Q, r, W[:r], W[r:], ell


VARIANTS = ("OrthS", "InS", "In", "OrthS-rand")


def factorize(prob_rowptr, prob_colind, prob_vals, tree: Tree, eps: float, skip: int = 0,
              trace: Optional[list] = None, variant: str = "OrthS", sketch=None,
              order: str = "coloured") -> Factor:
    """Algorithm 2.  ``trace`` (a list, tests only) receives (step, phase,
    set of block keys) before and after each level's sparsification.
    ``variant``: "OrthS" (Algorithm 2), "InS" or "In" (Sec. 4.3 ablation:
    interpolative transformations with / without the block scaling), or
    "OrthS-rand" (OrthS with the randomized range finder); the latter needs
    ``sketch(step, cluster, m, ell)`` returning an m x ell Gaussian matrix."""
    if variant not in VARIANTS:
        raise ValueError(f"unknown variant {variant!r}")
    if variant == "OrthS-rand" and sketch is None:
        raise ValueError("the randomized variant needs a sketch generator")
    if order not in ("coloured", "simultaneous") or (order == "simultaneous" and variant != "OrthS"):
        raise ValueError(f"order {order!r} is not available for variant {variant!r}")
    n, L = tree.n, tree.L
    rowptr = np.asarray(prob_rowptr, dtype=np.int64)
    colind = np.asarray(prob_colind, dtype=np.int64)
    vals = np.asarray(prob_vals, dtype=np.float64)
    pos = np.empty(n, dtype=np.int64)
    pos[tree.perm] = np.arange(n)
    nc = tree.keys.shape[0]
    cl_of_pos = np.repeat(np.arange(nc), np.diff(tree.cluster_ptr))
    # initial dense blocks from A (in permuted positions)
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    pi, pj = pos[rows], pos[colind]
    ci, cj = cl_of_pos[pi], cl_of_pos[pj]
    li = pi - tree.cluster_ptr[ci]
    lj = pj - tree.cluster_ptr[cj]
    size = np.diff(tree.cluster_ptr).astype(np.int64)
    blocks: Dict[Tuple[int, int], np.ndarray] = {}
    for x, y, a, b, v in zip(ci, cj, li, lj, vals):
        key = (int(x), int(y))
        blk = blocks.get(key)
        if blk is None:
            blk = blocks[key] = np.zeros((size[x], size[y]))
        blk[a, b] += v
    slots = [np.arange(tree.cluster_ptr[i], tree.cluster_ptr[i + 1]) for i in range(nc)]
    F = Factor()

    def nbrs_of(p):
        return sorted(q for (a, q) in blocks if a == p and q != p)

    for t, st in enumerate(tree.steps, start=1):
        nt = st.keys.shape[0]
        F.sizes_before.append(size.copy())
        # ---- eliminate every separator of this level (Sec. 2.4)
        for s in range(nt):
            if not st.elim[s]:
                continue
            if t == L:
                F.size_top = int(size[s])
            nb = nbrs_of(s)
            if size[s] == 0:
                Ls = np.zeros((0, 0))
                Xt = {q: np.zeros((0, size[q])) for q in nb}
            else:
                try:
                    Ls = np.linalg.cholesky(blocks[(s, s)])
                except np.linalg.LinAlgError as e:
                    raise NotSPDError(f"step {t} cluster {s}") from e
                Xt = {q: sla.solve_triangular(Ls, blocks[(s, q)], lower=True) for q in nb}
            for a in nb:
                for b in nb:
                    upd = Xt[a].T @ Xt[b]
                    if (a, b) in blocks:
                        blocks[(a, b)] = blocks[(a, b)] - upd
                    else:
                        blocks[(a, b)] = -upd
            for key in [k for k in blocks if s in k]:
                del blocks[key]
            F.ops.append(("E", slots[s], Ls, [(slots[q], Xt[q]) for q in nb]))
            F.mem_f += int(size[s] * (size[s] + 1) // 2 + size[s] * sum(size[q] for q in nb))
        rem = [i for i in range(nt) if not st.elim[i]]
        # sanity: the block pattern equals the symbolic fill pattern
        for p in rem:
            if nbrs_of(p) != st.adjf[p]:
                raise RuntimeError("numeric pattern differs from the symbolic one")
        ranks = {}
        if skip < t < L:
            # ---- scale every interface (Sec. 2.5); the In variant skips it
            Lp = {}
            for p in (rem if variant != "In" else []):
                if size[p] == 0:
                    Lp[p] = np.zeros((0, 0))
                    continue
                try:
                    Lp[p] = np.linalg.cholesky(blocks[(p, p)])
                except np.linalg.LinAlgError as e:
                    raise NotSPDError(f"scaling step {t} cluster {p}") from e
            for p in (rem if variant != "In" else []):
                for q in st.adjf[p]:
                    if p < q:
                        X = sla.solve_triangular(Lp[p], blocks[(p, q)], lower=True) if size[p] else blocks[(p, q)]
                        if size[q]:
                            X = sla.solve_triangular(Lp[q], X.T, lower=True).T
                        blocks[(p, q)] = X
                        blocks[(q, p)] = X.T.copy()
            for p in (rem if variant != "In" else []):
                blocks[(p, p)] = np.eye(size[p])
                F.ops.append(("S", slots[p], Lp[p]))
                F.mem_f += int(size[p] * (size[p] + 1) // 2)
            # ---- sparsify every interface, colour by colour (Sec. 2.6.1)
            if trace is not None:
                trace.append((t, "pre", frozenset(blocks)))
            ncol = int(st.colour.max()) + 1 if rem else 0
            if order == "simultaneous":
                # all interfaces from the same scaled matrix, then the
                # two-sided transform of every coupling block
                Qs = {}
                for p in rem:
                    nb = st.adjf[p]
                    if not nb:
                        continue
                    Apn = np.hstack([blocks[(p, q)] for q in nb])
                    Q, r, _, _ = sparsify_interface(Apn, eps)
                    Qs[p] = (Q, r)
                for (a, b_) in list(blocks):
                    if a != b_ and a < b_:
                        Qa, ra = Qs[a]
                        Qb, rb = Qs[b_]
                        X = Qa[:, :ra].T @ blocks[(a, b_)] @ Qb[:, :rb]
                        blocks[(a, b_)] = X
                        blocks[(b_, a)] = X.T.copy()
                for p in rem:
                    if p not in Qs:
                        continue
                    Q, r = Qs[p]
                    blocks[(p, p)] = np.eye(r)
                    F.ops.append(("Q", slots[p], Q))
                    pz = int(size[p])
                    F.mem_f += int(r * pz - r * (r + 1) // 2 + r)
                    ranks[p] = r
                    size[p] = r
                    slots[p] = slots[p][:r]
                ncol = 0
            for c in range(ncol):
                for p in rem:
                    if st.colour[p] != c:
                        continue
                    nb = st.adjf[p]
                    if not nb:
                        continue
                    widths = [int(size[q]) for q in nb]
                    if variant in ("InS", "In"):
                        Anp = np.vstack([blocks[(q, p)] for q in nb])
                        cl, fl, T, Lf, Xfc, Acc, _ = sparsify_interface_interp(Anp, blocks[(p, p)], eps)
                        r = int(cl.size)
                        for q in nb:  # A_qc is a subset of A_qp; A_qf - A_qc T_cf is dropped
                            blocks[(q, p)] = blocks[(q, p)][:, cl].copy()
                            blocks[(p, q)] = blocks[(q, p)].T.copy()
                        blocks[(p, p)] = Acc
                        cs, fs = slots[p][cl], slots[p][fl]
                        if fl.size:
                            F.ops.append(("T", cs, fs, T))
                            F.ops.append(("E", fs, Lf, [(cs, Xfc)]))
                            F.mem_f += int(r * fl.size * 2 + fl.size * (fl.size + 1) // 2)
                        ranks[p] = r
                        size[p] = r
                        slots[p] = cs
                        continue
                    Apn = np.hstack([blocks[(p, q)] for q in nb]) if nb else np.zeros((size[p], 0))
                    if variant == "OrthS-rand":
                        m = Apn.shape[1]
                        Om = sketch(t, p, m, min(int(size[p]), m))
                        Q, r, Wc, _, _ = sparsify_interface_rand(Apn, eps, Om)
                    else:
                        Q, r, Wc, _ = sparsify_interface(Apn, eps)
                    off = 0
                    for q, w in zip(nb, widths):
                        blocks[(p, q)] = Wc[:, off:off + w].copy()
                        blocks[(q, p)] = Wc[:, off:off + w].T.copy()
                        off += w
                    blocks[(p, p)] = np.eye(r)
                    F.ops.append(("Q", slots[p], Q))
                    pz = int(size[p])
                    F.mem_f += int(r * pz - r * (r + 1) // 2 + r)
                    ranks[p] = r
                    size[p] = r
                    slots[p] = slots[p][:r]
            if trace is not None:
                trace.append((t, "post", frozenset(blocks)))
        F.ranks.append(ranks)
        after = size.copy()
        after[st.elim == 1] = 0
        F.sizes_after.append(after)
        if t == L:
            break
        # ---- merge (Sec. 2.7)
        nxt = tree.steps[t]
        pof = {}
        for P, ch in enumerate(nxt.children):
            for c in ch:
                pof[c] = P
        new_size = np.array([sum(int(size[c]) for c in ch) for ch in nxt.children], dtype=np.int64)
        coff = {}
        for P, ch in enumerate(nxt.children):
            o = 0
            for c in ch:
                coff[c] = o
                o += int(size[c])
        nb_new: Dict[Tuple[int, int], np.ndarray] = {}
        for (a, b), blk in blocks.items():
            P, Q = pof[a], pof[b]
            tgt = nb_new.get((P, Q))
            if tgt is None:
                tgt = nb_new[(P, Q)] = np.zeros((new_size[P], new_size[Q]))
            tgt[coff[a]:coff[a] + blk.shape[0], coff[b]:coff[b] + blk.shape[1]] = blk
        for P in range(len(nxt.children)):
            if (P, P) not in nb_new:
                nb_new[(P, P)] = np.zeros((new_size[P], new_size[P]))
        slots = [np.concatenate([slots[c] for c in ch]) if ch else np.zeros(0, np.int64) for ch in nxt.children]
        blocks = nb_new
        size = new_size
    return F


# --------------------------------------------------------------------------
# preconditioner apply  z = M M^T r  (Sec. 2.8)
# --------------------------------------------------------------------------

def apply(F: Factor, r: np.ndarray) -> np.ndarray:
    v = np.array(r, dtype=np.float64, copy=True)
    for op in F.ops:                       # forward: leaves -> root
        if op[0] == "E":
            _, ss, Ls, nbl = op
            if ss.size:
                y = sla.solve_triangular(Ls, v[ss], lower=True)
                v[ss] = y
                for ns, Xt in nbl:
                    v[ns] -= Xt.T @ y
        elif op[0] == "S":
            _, ps, Lp = op
            if ps.size:
                v[ps] = sla.solve_triangular(Lp, v[ps], lower=True)
        elif op[0] == "T":                 # v <- T_p^T v
            _, cs, fs, T = op
            v[fs] -= T.T @ v[cs]
        else:
            _, ps, Q = op
            v[ps] = Q.T @ v[ps]
    for op in reversed(F.ops):             # backward: root -> leaves
        if op[0] == "E":
            _, ss, Ls, nbl = op
            if ss.size:
                acc = v[ss].copy()
                for ns, Xt in nbl:
                    acc -= Xt @ v[ns]
                v[ss] = sla.solve_triangular(Ls, acc, lower=True, trans="T")
        elif op[0] == "S":
            _, ps, Lp = op
            if ps.size:
                v[ps] = sla.solve_triangular(Lp, v[ps], lower=True, trans="T")
        elif op[0] == "T":                 # v <- T_p v
            _, cs, fs, T = op
            v[cs] -= T @ v[fs]
        else:
            _, ps, Q = op
            v[ps] = Q @ v[ps]
    return v


def permuted_matrix(rowptr, colind, vals, perm):
    """P A P^T as scipy CSR (positions in the cluster order)."""
    import scipy.sparse as sp
    n = perm.size
    A = sp.csr_matrix((np.asarray(vals, np.float64), np.asarray(colind, np.int64), np.asarray(rowptr, np.int64)),
                      shape=(n, n))
    return A[perm][:, perm].tocsr()


def pcg(A, b: np.ndarray, prec, tol: float = 1e-10, maxit: int = 500):
    """Preconditioned CG; returns (x, iterations, true relative residual)."""
    b = np.asarray(b, dtype=np.float64)
    nb = float(np.linalg.norm(b))
    x = np.zeros_like(b)
    if nb == 0.0:
        return x, 0, 0.0
    r = b.copy()
    z = prec(r)
    p = z.copy()
    rz = float(r @ z)
    it = 0
    while it < maxit:
        q = A @ p
        alpha = rz / float(p @ q)
        x += alpha * p
        r -= alpha * q
        it += 1
        if np.linalg.norm(r) / nb <= tol:
            rt = b - A @ x
            if np.linalg.norm(rt) / nb <= tol:
                break
            r = rt
            z = prec(r)
            p = z.copy()
            rz = float(r @ z)
            continue
        z = prec(r)
        rz_new = float(r @ z)
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
    return x, it, float(np.linalg.norm(b - A @ x) / nb)


@dataclass
class Result:
    x: np.ndarray
    iters: int
    relres: float
    tree: Tree
    factor: Factor


def solve(prob, b, L: int, eps: float, skip: int = 0, tol: float = 1e-10, maxit: int = 500,
          use_coords: bool = True, variant: str = "OrthS", sketch=None, order: str = "coloured") -> Result:
    """analyze + factorize + PCG on the original ordering of b / x."""
    coords = prob.coords if use_coords else None
    tree = analyze(prob.n, prob.rowptr, prob.colind, coords, L)
    F = factorize(prob.rowptr, prob.colind, prob.vals, tree, eps, skip, variant=variant, sketch=sketch, order=order)
    Ap = permuted_matrix(prob.rowptr, prob.colind, prob.vals, tree.perm)
    xp, it, rr = pcg(Ap, np.asarray(b)[tree.perm], lambda r: apply(F, r), tol, maxit)
    x = np.empty(prob.n)
    x[tree.perm] = xp
    return Result(x, it, rr, tree, F)


# --------------------------------------------------------------------------
# flat integer view of the analysis (same layout as the C-ABI queries)
# --------------------------------------------------------------------------

def flat_tree(tree: Tree) -> dict:
    out = {
        "perm": tree.perm.astype(np.int32),
        "cluster_ptr": tree.cluster_ptr.astype(np.int32),
        "keys": tree.keys.astype(np.int32).reshape(-1),
    }
    for t, st in enumerate(tree.steps, start=1):
        nt = st.keys.shape[0]
        cptr = np.zeros(nt + 1, dtype=np.int32)
        cptr[1:] = np.cumsum([len(c) for c in st.children])
        aptr = np.zeros(nt + 1, dtype=np.int32)
        aptr[1:] = np.cumsum([len(a) for a in st.adj])
        fptr = np.zeros(nt + 1, dtype=np.int32)
        fptr[1:] = np.cumsum([len(a) for a in st.adjf])
        cat = lambda ls: np.array([v for l in ls for v in l], dtype=np.int32)
        out[f"step{t}"] = {
            "keys": st.keys.astype(np.int32).reshape(-1),
            "child_ptr": cptr, "child_idx": cat(st.children),
            "elim": st.elim.astype(np.int32), "colour": st.colour.astype(np.int32),
            "adj_ptr": aptr, "adj_idx": cat(st.adj),
            "adjf_ptr": fptr, "adjf_idx": cat(st.adjf),
        }
    return out


def dense_preconditioner(F: Factor, n: int) -> np.ndarray:
    """M M^T as a dense matrix (tiny cases only)."""
    return np.column_stack([apply(F, e) for e in np.eye(n)])

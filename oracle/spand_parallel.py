"""All-core timing leg of the FP64 oracle.

TEST INFRASTRUCTURE ONLY, like ``spand_oracle``: only ``tests/`` and
``bench.py`` (its CPU-baseline legs) may import or run this module; the
product path never does.

``factorize`` is Algorithm 2 (OrthS, coloured order) exactly as
``spand_oracle.factorize`` computes it, with the independent block work of
each level spread over a process pool:

* eliminate (Sec. 2.4): the separators of one level are never adjacent, so
  L_s = chol(A_ss), X_sq = L_s^{-1} A_sq and the products X_sa^T X_sb run in
  parallel, one task per separator; the updates are then subtracted from the
  target blocks in the serial oracle's order (separators ascending);
* scale (Sec. 2.5): one task per interface for L_p = chol(A_pp), then one
  task per adjacent pair for L_p^{-1} A_pq L_q^{-T};
* sparsify (Sec. 2.6.1): the interfaces of one colour are pairwise
  non-adjacent, so their column-pivoted QRs (``spand_oracle.
  sparsify_interface``) run in parallel, one task per interface, colours in
  sequence; the write-back of W_cn follows in the main process;
* merge (Sec. 2.7): in the main process, as in the serial oracle.

The pool is started with the ``spawn`` method (the workers import this
module and the oracle afresh).  Blocks travel to the workers and back by
pickling; each worker's BLAS/LAPACK uses one thread (the parent's
OPENBLAS/OMP/MKL thread variables, which the caller sets).  The apply and
PCG stay serial (``spand_oracle.apply`` / ``pcg``): the apply walks the
dependent transforms of Sec. 2.8 in order.

The result equals the serial oracle's in ranks and operators up to the
rounding of X_sb^T X_sa, formed here as the transpose of X_sa^T X_sb.
"""
from __future__ import annotations

import multiprocessing as mp
from concurrent.futures import ProcessPoolExecutor
from typing import Dict, List, Tuple

import numpy as np
import scipy.linalg as sla

from oracle import spand_oracle as O


def make_pool(workers: int) -> ProcessPoolExecutor:
    """A pool of `workers` processes started with `spawn`."""
    return ProcessPoolExecutor(max_workers=int(workers), mp_context=mp.get_context("spawn"))


# ---- worker tasks (module level: picklable by reference)

def _elim_task(args):
    """One separator s (Sec. 2.4): L_s, X_sq = L_s^{-1} A_sq for every
    neighbour q, and the Schur products X_sa^T X_sb for a <= b (neighbour
    list positions).  Returns (s, L_s, [X_sq], {(i, j): X_si^T X_sj}) or
    (s, None, ...) when A_ss is not SPD."""
    s, Ass, Asq = args
    n = Ass.shape[0]
    if n == 0:
        Xt = [np.zeros((0, A.shape[1])) for A in Asq]
        Ls = np.zeros((0, 0))
    else:
        try:
            Ls = np.linalg.cholesky(Ass)
        except np.linalg.LinAlgError:
            return s, None, None, None
        Xt = [sla.solve_triangular(Ls, A, lower=True) for A in Asq]
    upd = {}
    for i in range(len(Xt)):
        for j in range(i, len(Xt)):
            upd[(i, j)] = Xt[i].T @ Xt[j]
    return s, Ls, Xt, upd


def _chol_task(args):
    """L_p = chol(A_pp) of one interface (Sec. 2.5); None when not SPD."""
    p, App = args
    if App.shape[0] == 0:
        return p, np.zeros((0, 0))
    try:
        return p, np.linalg.cholesky(App)
    except np.linalg.LinAlgError:
        return p, None


def _scale_pair_task(args):
    """A_pq <- L_p^{-1} A_pq L_q^{-T} for one adjacent pair p < q (Sec. 2.5)."""
    key, Lp, Lq, Apq = args
    X = sla.solve_triangular(Lp, Apq, lower=True) if Lp.shape[0] else Apq
    if Lq.shape[0]:
        X = sla.solve_triangular(Lq, X.T, lower=True).T
    return key, X


def _sparsify_task(args):
    """The column-pivoted QR of one scaled interface (Sec. 2.6.1)."""
    p, Apn, eps = args
    Q, r, Wc, _ = O.sparsify_interface(Apn, eps)
    return p, Q, r, Wc


def _map(pool, fn, items, workers):
    if not items:
        return []
    chunk = max(1, len(items) // (4 * workers))
    return list(pool.map(fn, items, chunksize=chunk))


def factorize(prob_rowptr, prob_colind, prob_vals, tree: O.Tree, eps: float, pool: ProcessPoolExecutor,
              workers: int, skip: int = 0) -> O.Factor:
    """Algorithm 2 (OrthS, coloured order) with the block work of each level
    on `pool` (see the module docstring); returns the oracle's Factor."""
    n, L = tree.n, tree.L
    rowptr = np.asarray(prob_rowptr, dtype=np.int64)
    colind = np.asarray(prob_colind, dtype=np.int64)
    vals = np.asarray(prob_vals, dtype=np.float64)
    pos = np.empty(n, dtype=np.int64)
    pos[tree.perm] = np.arange(n)
    nc = tree.keys.shape[0]
    cl_of_pos = np.repeat(np.arange(nc), np.diff(tree.cluster_ptr))
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
    F = O.Factor()
    for t, st in enumerate(tree.steps, start=1):
        nt = st.keys.shape[0]
        F.sizes_before.append(size.copy())
        # ---- eliminate (Sec. 2.4): one task per separator of the level
        nbl: Dict[int, List[int]] = {}
        for (a, q) in blocks:
            if a != q and st.elim[a]:
                nbl.setdefault(a, []).append(q)
        seps = [s for s in range(nt) if st.elim[s]]
        for s in seps:
            nbl[s] = sorted(nbl.get(s, []))
        res = _map(pool, _elim_task, [(s, blocks[(s, s)], [blocks[(s, q)] for q in nbl[s]]) for s in seps], workers)
        for s, Ls, Xt, upd in res:
            if Ls is None:
                raise O.NotSPDError(f"step {t} cluster {s}")
            if t == L:
                F.size_top = int(size[s])
            nb = nbl[s]
            for i, a in enumerate(nb):
                for j, b in enumerate(nb):
                    u = upd[(i, j)] if i <= j else upd[(j, i)].T
                    blocks[(a, b)] = blocks[(a, b)] - u if (a, b) in blocks else -u
            F.ops.append(("E", slots[s], Ls, [(slots[q], Xt[k]) for k, q in enumerate(nb)]))
            F.mem_f += int(size[s] * (size[s] + 1) // 2 + size[s] * sum(size[q] for q in nb))
        for key in [k for k in blocks if st.elim[k[0]] or st.elim[k[1]]]:
            del blocks[key]
        rem = [i for i in range(nt) if not st.elim[i]]
        ranks = {}
        if skip < t < L:
            # ---- scale (Sec. 2.5)
            Lp = {}
            for p, Lc in _map(pool, _chol_task, [(p, blocks[(p, p)]) for p in rem], workers):
                if Lc is None:
                    raise O.NotSPDError(f"scaling step {t} cluster {p}")
                Lp[p] = Lc
            pairs = [((p, q), Lp[p], Lp[q], blocks[(p, q)]) for p in rem for q in st.adjf[p] if p < q]
            for (p, q), X in _map(pool, _scale_pair_task, pairs, workers):
                blocks[(p, q)] = X
                blocks[(q, p)] = X.T.copy()
            for p in rem:
                blocks[(p, p)] = np.eye(size[p])
                F.ops.append(("S", slots[p], Lp[p]))
                F.mem_f += int(size[p] * (size[p] + 1) // 2)
            # ---- sparsify (Sec. 2.6.1), colour by colour
            ncol = int(st.colour.max()) + 1 if rem else 0
            for c in range(ncol):
                todo = [p for p in rem if st.colour[p] == c and st.adjf[p]]
                items = [(p, np.hstack([blocks[(p, q)] for q in st.adjf[p]]), eps) for p in todo]
                for p, Q, r, Wc in _map(pool, _sparsify_task, items, workers):
                    off = 0
                    for q in st.adjf[p]:
                        w = int(size[q])
                        blocks[(p, q)] = Wc[:, off:off + w].copy()
                        blocks[(q, p)] = Wc[:, off:off + w].T.copy()
                        off += w
                    blocks[(p, p)] = np.eye(r)
                    F.ops.append(("Q", slots[p], Q))
                    F.mem_f += int(r * int(size[p]) - r * (r + 1) // 2 + r)
                    ranks[p] = r
                    size[p] = r
                    slots[p] = slots[p][:r]
        F.ranks.append(ranks)
        after = size.copy()
        after[st.elim == 1] = 0
        F.sizes_after.append(after)
        if t == L:
            break
        # ---- merge (Sec. 2.7)
        nxt = tree.steps[t]
        pof, coff = {}, {}
        for P, ch in enumerate(nxt.children):
            o = 0
            for ch_i in ch:
                pof[ch_i] = P
                coff[ch_i] = o
                o += int(size[ch_i])
        new_size = np.array([sum(int(size[ch_i]) for ch_i in ch) for ch in nxt.children], dtype=np.int64)
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
        slots = [np.concatenate([slots[ch_i] for ch_i in ch]) if ch else np.zeros(0, np.int64)
                 for ch in nxt.children]
        blocks = nb_new
        size = new_size
    return F

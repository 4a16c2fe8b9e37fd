// Batched kernels of the level-by-level spaND factorization (Algorithm 2).
// Every kernel processes all clusters of one step (or one colour) in a single
// launch; descriptors are built by the host scheduler once the step's block
// sizes are known.
#pragma once

#include "dense_tiles.cuh"

namespace spand {

// ---------------------------------------------------------------- descriptors

template <typename T>
struct RowDesc {      // a cluster's block row or its diagonal block
  T* R;               // column-major, leading dimension ld
  int32_t n;          // rows (cluster size)
  int32_t ld;
};

template <typename T>
struct TrsmTask {     // X = U^{-T} B for columns [c0, c1) of a block row (U = its diag block)
  T* R;
  int32_t n, ld, c0, c1;
};

template <typename T>
struct SchurBlock {   // target block (a, b), a <= b, of the elimination update (Sec. 2.4)
  T* C1;              // block (a, b) in a's row: rows |a|, cols |b|
  T* C2;              // block (b, a) in b's row (nullptr when a == b)
  int32_t ld1, ld2, rows, cols;
  int32_t cbeg, cend; // contributors
};

template <typename T>
struct SchurContrib { // one eliminated separator s adjacent to both a and b
  const T* Xa;        // X^T columns of a inside s's row: Xa[k + i*lds], k < ns
  const T* Xb;
  int32_t lds, ns;
};

struct SchurTile {
  int32_t block, i0, j0;
};

template <typename T>
struct CopyTask {     // dst[r + c*ldd] = src[r + c*lds] (trans = 0) or src[c + r*lds] (trans = 1)
  const T* src;
  T* dst;
  int32_t lds, ldd, rows, cols, trans, pad;
};

struct CopyTile {
  int32_t task, r0, c0;
};

template <typename T>
struct CpqrNbr {      // neighbour q of p in the sparsified row A_pn (Sec. 2.6.1)
  T* Rq;              // q's block row (leading dimension ldq)
  int32_t q, off_pq, off_qp, ldq;
};

template <typename T>
struct CpqrTask {
  T* Rp;              // p's block row
  T* work;            // |p| x m_max workspace
  T* norms;           // m_max
  int32_t* piv;       // m_max
  T* Qc;              // |p| x |p| capacity (first r columns = Q_pc on exit)
  int32_t p, np, ldp, nbeg, nend, m_max;
};

// ---------------------------------------------------------------- assembly

// Scatter A's values into the step-1 block rows: rows[dst_row[e]][dst_off[e]] = vals[e].
template <typename T>
__global__ void k_assemble(const double* __restrict__ vals, const int32_t* __restrict__ dst_row,
                           const int64_t* __restrict__ dst_off, T* const* __restrict__ rows, int64_t nnz) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = dst_row[e];
    if (r >= 0) rows[r][dst_off[e]] = (T)vals[e];
  }
}

// ---------------------------------------------------------------- tiled Cholesky

// Tile step k, phase 1: factor diagonal tile (k, k) of every block.
template <typename T>
__global__ void __launch_bounds__(NT) k_potrf_diag(const RowDesc<T>* __restrict__ rows, int k, int* info) {
  extern __shared__ __align__(16) unsigned char smraw[];
  SqTile<T>& s = *reinterpret_cast<SqTile<T>*>(smraw);
  const RowDesc<T> d = rows[blockIdx.x];
  const int k0 = k * TB;
  if (k0 >= d.n) return;
  const int nb = min(TB, d.n - k0);
  T* P = d.R + k0 + (size_t)k0 * d.ld;
  load_tile(s, P, d.ld, nb, nb);
  __syncthreads();
  const bool ok = potrf_tile_upper(s, nb);
  if (!ok) {
    if (threadIdx.x == 0) atomicCAS(info, 0, (int)blockIdx.x + 1);
    return;
  }
  store_tile(s, P, d.ld, nb, nb);
}

// Tile step k, phase 2: U_kj = U_kk^{-T} A_kj for the tiles j > k of the diagonal block.
template <typename T>
__global__ void __launch_bounds__(NT) k_potrf_trsm(const RowDesc<T>* __restrict__ rows, int k) {
  extern __shared__ __align__(16) unsigned char smraw[];
  SqTile<T>& U = *reinterpret_cast<SqTile<T>*>(smraw);
  SqTile<T>& B = *reinterpret_cast<SqTile<T>*>(smraw + sizeof(SqTile<T>));
  const RowDesc<T> d = rows[blockIdx.y];
  const int k0 = k * TB;
  const int j0 = k0 + TB * (1 + blockIdx.x);
  if (j0 >= d.n) return;
  const int nb = min(TB, d.n - k0), nc = min(TB, d.n - j0);
  load_tile(U, d.R + k0 + (size_t)k0 * d.ld, d.ld, nb, nb);
  load_tile(B, d.R + k0 + (size_t)j0 * d.ld, d.ld, nb, nc);
  __syncthreads();
  trsm_tile_upperT(U, B, nb, nc);
  store_tile(B, d.R + k0 + (size_t)j0 * d.ld, d.ld, nb, nc);
}

// Tile step k, phase 3: A_ij -= U_ki^T U_kj for k < i <= j (upper trailing tiles).
template <typename T>
__global__ void __launch_bounds__(NT) k_potrf_update(const RowDesc<T>* __restrict__ rows, int k) {
  __shared__ TileSmem<T> sm;
  const RowDesc<T> d = rows[blockIdx.y];
  const int nt = (d.n + TB - 1) / TB;
  const int m = nt - k - 1;  // trailing tiles per side
  if (m <= 0) return;
  int lin = blockIdx.x;
  if (lin >= m * (m + 1) / 2) return;
  // decode lin -> (i, j) with i <= j, row-wise over the upper triangle
  int i = 0;
  while (lin >= m - i) { lin -= m - i; ++i; }
  const int j = i + lin;
  const int i0 = (k + 1 + i) * TB, j0 = (k + 1 + j) * TB, k0 = k * TB;
  const int mi = min(TB, d.n - i0), nj = min(TB, d.n - j0), kb = min(TB, d.n - k0);
  T acc[4][4];
  zero_acc(acc);
  tn_acc(acc, d.R + k0 + (size_t)i0 * d.ld, d.ld, mi, d.R + k0 + (size_t)j0 * d.ld, d.ld, nj, kb, sm);
  sub_store(acc, d.R + i0 + (size_t)j0 * d.ld, d.ld, mi, nj);
}

// X = U^{-T} B for one 64-column panel of a block row: left-looking over the
// row tiles (B_i -= sum_{l<i} U_li^T X_l; X_i = U_ii^{-T} B_i).
template <typename T>
__global__ void __launch_bounds__(NT) k_trsm_cols(const TrsmTask<T>* __restrict__ tasks) {
  extern __shared__ __align__(16) unsigned char smraw[];
  SqTile<T>& U = *reinterpret_cast<SqTile<T>*>(smraw);
  SqTile<T>& B = *reinterpret_cast<SqTile<T>*>(smraw + sizeof(SqTile<T>));
  TileSmem<T>& sm = *reinterpret_cast<TileSmem<T>*>(smraw + 2 * sizeof(SqTile<T>));
  const TrsmTask<T> d = tasks[blockIdx.x];
  const int nc = d.c1 - d.c0;
  if (nc <= 0 || d.n <= 0) return;
  T* X = d.R + (size_t)d.c0 * d.ld;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int i0 = 0; i0 < d.n; i0 += TB) {
    const int nb = min(TB, d.n - i0);
    T acc[4][4];
    zero_acc(acc);
    if (i0 > 0) tn_acc(acc, d.R + (size_t)i0 * d.ld, d.ld, nb, X, d.ld, nc, i0, sm);
    load_tile(U, d.R + i0 + (size_t)i0 * d.ld, d.ld, nb, nb);
    load_tile(B, X + i0, d.ld, nb, nc);
    __syncthreads();
#pragma unroll
    for (int ii = 0; ii < 4; ++ii)
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        const int r = tx + 16 * ii, c = ty + 16 * jj;
        B.v[r][c] -= acc[ii][jj];
      }
    __syncthreads();
    trsm_tile_upperT(U, B, nb, nc);
    store_tile(B, X + i0, d.ld, nb, nc);
    __syncthreads();
  }
}

// ---------------------------------------------------------------- Schur update

// Pull form of A_{ab} -= sum_s X_{as} X_{bs}^T over the separators s adjacent
// to both a and b (Sec. 2.4), one 64x64 output tile per CTA, contributors in a
// fixed order (deterministic, no atomics).  Writes block (a,b) in a's row and
// its transpose (b,a) in b's row.
template <typename T>
__global__ void __launch_bounds__(NT) k_schur(const SchurTile* __restrict__ tiles,
                                             const SchurBlock<T>* __restrict__ blocks,
                                             const SchurContrib<T>* __restrict__ contribs) {
  __shared__ TileSmem<T> sm;
  const SchurTile t = tiles[blockIdx.x];
  const SchurBlock<T> b = blocks[t.block];
  const int mi = min(TB, b.rows - t.i0), nj = min(TB, b.cols - t.j0);
  T acc[4][4];
  zero_acc(acc);
  for (int c = b.cbeg; c < b.cend; ++c) {
    const SchurContrib<T> s = contribs[c];
    if (s.ns <= 0) continue;
    tn_acc(acc, s.Xa + (size_t)t.i0 * s.lds, s.lds, mi, s.Xb + (size_t)t.j0 * s.lds, s.lds, nj, s.ns, sm);
  }
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int jj = 0; jj < 4; ++jj) {
    const int c = ty + 16 * jj;
    if (c >= nj) continue;
#pragma unroll
    for (int ii = 0; ii < 4; ++ii) {
      const int r = tx + 16 * ii;
      if (r >= mi) continue;
      const size_t o1 = (size_t)(t.i0 + r) + (size_t)(t.j0 + c) * b.ld1;
      const T v = b.C1[o1] - acc[ii][jj];
      b.C1[o1] = v;
      if (b.C2) b.C2[(size_t)(t.j0 + c) + (size_t)(t.i0 + r) * b.ld2] = v;
    }
  }
}

// ---------------------------------------------------------------- copies

template <typename T>
__global__ void __launch_bounds__(NT) k_copy(const CopyTile* __restrict__ tiles, const CopyTask<T>* __restrict__ tasks) {
  __shared__ T s[32][33];
  const CopyTile t = tiles[blockIdx.x];
  const CopyTask<T> d = tasks[t.task];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  if (!d.trans) {
    for (int c = ty; c < 32; c += 8) {
      const int rr = t.r0 + tx, cc = t.c0 + c;
      if (rr < d.rows && cc < d.cols) d.dst[rr + (size_t)cc * d.ldd] = d.src[rr + (size_t)cc * d.lds];
    }
    return;
  }
  // dst (rows x cols) = transpose of src (cols x rows)
  for (int c = ty; c < 32; c += 8) {   // read src rows = dst cols
    const int sr = t.c0 + tx, sc = t.r0 + c;
    if (sr < d.cols && sc < d.rows) s[c][tx] = d.src[sr + (size_t)sc * d.lds];
  }
  __syncthreads();
  for (int c = ty; c < 32; c += 8) {
    const int rr = t.r0 + tx, cc = t.c0 + c;
    if (rr < d.rows && cc < d.cols) d.dst[rr + (size_t)cc * d.ldd] = s[tx][c];
  }
}

// Diagonal block <- identity (after scaling, Sec. 2.5: S_p A S_p^T has I on p).
template <typename T>
__global__ void k_set_identity(const RowDesc<T>* __restrict__ rows, int nrows) {
  const RowDesc<T> d = rows[blockIdx.y];
  const int64_t tot = (int64_t)d.n * d.n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % d.n), j = (int)(e / d.n);
    d.R[i + (size_t)j * d.ld] = (i == j) ? T(1) : T(0);
  }
}

// ---------------------------------------------------------------- sparsification

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Orthogonal sparsification of one scaled interface p (Sec. 2.6.1), one CTA:
//   gather A_pn (all current neighbour columns, in neighbour order) ->
//   Householder QR with column pivoting (largest remaining column norm, lowest
//   index on ties; norms recomputed exactly after every reflector) ->
//   stop at the first k with |R_kk| < eps |R_00| (truncation rule of Sec. 4) ->
//   write W_cn = R[0:r, :] P^T into p's row and its transpose into the rows of
//   the neighbours, set A_cc = I, form Q_pc = H_0 ... H_{r-1} [I_r; 0].
// The fine dofs f are dropped (their coupling W_fn is O(eps)).
template <typename T>
__global__ void __launch_bounds__(NT) k_cpqr(const CpqrTask<T>* __restrict__ tasks,
                                            const int32_t* __restrict__ list,
                                            const CpqrNbr<T>* __restrict__ nbrs,
                                            int32_t* __restrict__ cur_size, T eps) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const CpqrTask<T> d = tasks[list[blockIdx.x]];
  const int np = d.np;
  const int nnb = d.nend - d.nbeg;
  // shared: cstart[nnb+1] ints, v[np] T, red scratch
  int* cstart = reinterpret_cast<int*>(smraw);
  T* sv = reinterpret_cast<T*>(smraw + ((sizeof(int) * (nnb + 1) + 15) & ~size_t(15)));
  __shared__ T red_v[NT / 32];
  __shared__ int red_i[NT / 32];
  __shared__ T s_beta, s_tau, s_r00;
  __shared__ int s_piv, s_stop;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = NT / 32;
  if (tid == 0) {
    int m = 0;
    for (int e = 0; e < nnb; ++e) {
      cstart[e] = m;
      m += cur_size[nbrs[d.nbeg + e].q];
    }
    cstart[nnb] = m;
  }
  __syncthreads();
  const int m = cstart[nnb];
  if (m == 0) {  // every neighbour already reduced to nothing: no coupling left, p is kept
    for (int64_t x = tid; x < (int64_t)np * np; x += NT) {
      const int i = (int)(x % np), j = (int)(x / np);
      d.Qc[i + (size_t)j * np] = (i == j) ? T(1) : T(0);
    }
    if (tid == 0) cur_size[d.p] = np;
    return;
  }
  T* W = d.work;  // np x m, ld = np
  // gather
  for (int e = 0; e < nnb; ++e) {
    const CpqrNbr<T> nb = nbrs[d.nbeg + e];
    const int w = cstart[e + 1] - cstart[e];
    const T* src = d.Rp + (size_t)nb.off_pq * d.ldp;
    T* dst = W + (size_t)cstart[e] * np;
    for (int64_t x = tid; x < (int64_t)np * w; x += NT) {
      const int i = (int)(x % np), j = (int)(x / np);
      dst[i + (size_t)j * np] = src[i + (size_t)j * d.ldp];
    }
  }
  __syncthreads();
  // column norms (squared) and identity pivots
  for (int j = warp; j < m; j += nw) {
    T s = 0;
    for (int i = lane; i < np; i += 32) {
      const T x = W[i + (size_t)j * np];
      s += x * x;
    }
    s = warp_sum(s);
    if (lane == 0) { d.norms[j] = s; d.piv[j] = j; }
  }
  __syncthreads();
  const int kmax = min(np, m);
  int r = kmax;
  for (int k = 0; k < kmax; ++k) {
    // pivot: argmax norms[j], j >= k (lowest j on ties)
    T best = T(-1);
    int bj = m;
    for (int j = k + tid; j < m; j += NT) {
      const T v = d.norms[j];
      if (v > best) { best = v; bj = j; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
      if (ov > best || (ov == best && oj < bj)) { best = ov; bj = oj; }
    }
    if (lane == 0) { red_v[warp] = best; red_i[warp] = bj; }
    __syncthreads();
    if (tid == 0) {
      T bv = red_v[0];
      int bi = red_i[0];
      for (int w = 1; w < nw; ++w)
        if (red_v[w] > bv || (red_v[w] == bv && red_i[w] < bi)) { bv = red_v[w]; bi = red_i[w]; }
      s_piv = (bi >= k && bi < m) ? bi : k;
    }
    __syncthreads();
    const int pj = s_piv;
    if (pj != k) {  // swap columns k and pj
      for (int i = tid; i < np; i += NT) {
        const T a = W[i + (size_t)k * np];
        W[i + (size_t)k * np] = W[i + (size_t)pj * np];
        W[i + (size_t)pj * np] = a;
      }
      if (tid == 0) {
        const T a = d.norms[k]; d.norms[k] = d.norms[pj]; d.norms[pj] = a;
        const int b = d.piv[k]; d.piv[k] = d.piv[pj]; d.piv[pj] = b;
      }
    }
    __syncthreads();
    // Householder vector of W[k:np, k]
    T s = 0;
    for (int i = k + 1 + tid; i < np; i += NT) {
      const T x = W[i + (size_t)k * np];
      s += x * x;
    }
    s = warp_sum(s);
    if (lane == 0) red_v[warp] = s;
    __syncthreads();
    if (tid == 0) {
      T sig = 0;
      for (int w = 0; w < nw; ++w) sig += red_v[w];
      const T alpha = W[k + (size_t)k * np];
      T beta, tau;
      if (sig == T(0)) {
        beta = alpha;
        tau = T(0);
      } else {
        const T nrm = sqrt(alpha * alpha + sig);
        beta = alpha >= T(0) ? -nrm : nrm;
        tau = (beta - alpha) / beta;
      }
      const T rkk = fabs(beta);
      if (k == 0) s_r00 = rkk;
      // prefix rule |R_kk| >= eps |R_00|; R_00 = 0 means A_pn = 0 (r = 0)
      s_stop = (s_r00 == T(0)) || (rkk < eps * s_r00);
      s_beta = beta;
      s_tau = tau;
      sv[k] = T(1);
    }
    __syncthreads();
    if (s_stop) { r = k; break; }
    const T beta = s_beta, tau = s_tau;
    const T alpha = W[k + (size_t)k * np];
    const T scal = (tau == T(0)) ? T(0) : T(1) / (alpha - beta);
    for (int i = k + 1 + tid; i < np; i += NT) {
      const T v = W[i + (size_t)k * np] * scal;
      W[i + (size_t)k * np] = v;
      sv[i] = v;
    }
    __syncthreads();
    if (tid == 0) {
      W[k + (size_t)k * np] = beta;
      d.norms[k] = tau;  // column k is done: keep tau where its norm was
    }
    // apply H = I - tau v v^T to columns j > k; refresh their trailing norms
    for (int j = k + 1 + warp; j < m; j += nw) {
      T* col = W + (size_t)j * np;
      T wdot = 0;
      for (int i = k + lane; i < np; i += 32) wdot += sv[i] * col[i];
      wdot = warp_sum(wdot) * tau;
      T nrm = 0;
      for (int i = k + lane; i < np; i += 32) {
        const T x = col[i] - wdot * sv[i];
        col[i] = x;
        if (i > k) nrm += x * x;
      }
      nrm = warp_sum(nrm);
      if (lane == 0) d.norms[j] = nrm;
    }
    __syncthreads();
  }
  // ---- write back W_cn = R[0:r, :] P^T into p's row and the transposes
  // column position j holds original column piv[j]
  for (int64_t x = tid; x < (int64_t)r * m; x += NT) {
    const int i = (int)(x % r), j = (int)(x / r);
    const T val = (j < r && i > j) ? T(0) : W[i + (size_t)j * np];
    const int oc = d.piv[j];
    // neighbour owning original column oc
    int lo = 0, hi = nnb - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (cstart[mid] <= oc) lo = mid; else hi = mid - 1;
    }
    const CpqrNbr<T> nb = nbrs[d.nbeg + lo];
    const int cc = oc - cstart[lo];
    d.Rp[i + (size_t)(nb.off_pq + cc) * d.ldp] = val;
    nb.Rq[cc + (size_t)(nb.off_qp + i) * nb.ldq] = val;
  }
  // A_cc = I
  for (int64_t x = tid; x < (int64_t)r * r; x += NT) {
    const int i = (int)(x % r), j = (int)(x / r);
    d.Rp[i + (size_t)j * d.ldp] = (i == j) ? T(1) : T(0);
  }
  __syncthreads();
  // Q_pc = H_0 H_1 ... H_{r-1} [I_r; 0]   (applied right to left)
  T* G = d.Qc;
  for (int64_t x = tid; x < (int64_t)np * r; x += NT) {
    const int i = (int)(x % np), j = (int)(x / np);
    G[i + (size_t)j * np] = (i == j) ? T(1) : T(0);
  }
  __syncthreads();
  for (int k = r - 1; k >= 0; --k) {
    const T tau = d.norms[k];
    if (tau != T(0)) {
      for (int j = k + warp; j < r; j += nw) {
        T* col = G + (size_t)j * np;
        T wdot = (lane == 0) ? col[k] : T(0);  // v_k[k] = 1
        for (int i = k + 1 + lane; i < np; i += 32) wdot += W[i + (size_t)k * np] * col[i];
        wdot = warp_sum(wdot);
        if (lane == 0) col[k] -= tau * wdot;
        for (int i = k + 1 + lane; i < np; i += 32) col[i] -= tau * wdot * W[i + (size_t)k * np];
      }
    }
    __syncthreads();
  }
  if (tid == 0) cur_size[d.p] = r;
}

}  // namespace spand

// Interpolative sparsification of interfaces (Sec. 2.6.2; the "InS" and "In"
// variants of the ablation of Sec. 4.3, with and without the block scaling of
// Sec. 2.5).  Per interface p of a colour, with A_np (m x np) the coupling of
// p to all its current neighbours:
//   1. the column-pivoted QR of A_np, A_np P = Q R, truncated by the rule of
//      Sec. 4 (keep k while |R_kk| >= eps |R_00|): computed through the Gram
//      matrix G = A_np^T A_np, whose diagonally pivoted Cholesky P^T G P =
//      R^T R picks the same pivots and the same R in exact arithmetic (the
//      largest remaining column norm of the QR is the largest remaining
//      diagonal of the Schur complement of G); c = the first r pivots, in
//      pivot order, f = the others in increasing order; r <= min(np, m);
//      the Gram route resolves |R_kk| only down to about sqrt(u) |R_00|
//      (below, its remaining diagonal is rounding), so at eps = 0 the
//      factorization is exact to about that level rather than to u;
//   2. T_cf = R_11^{-1} R_12 (r x |f|), so that A_nf = A_nc T_cf + O(eps);
//   3. with T_p = I - E_cf T_cf the diagonal block becomes
//        C_cf = A_cf - A_cc T_cf,
//        C_ff = A_ff - A_fc T_cf - T_cf^T C_cf
//      (= A_ff - A_fc T - T^T A_cf + T^T A_cc T; with the scaling, A_pp = I
//      and these are -T_cf and I + T_cf^T T_cf);
//   4. the coupling of p to its neighbours keeps the columns c (the dropped
//      A_nf - A_nc T_cf is O(eps)), A_cc stays, and the f dofs, now coupled
//      to c only, are eliminated next by the ordinary pivot Cholesky, block-
//      row solve and Schur kernels of Sec. 2.4 on the block row
//      [C_ff | C_fc] (C_ff = U_f^T U_f; a C_ff that is not positive definite
//      is the breakdown these variants can suffer).
// Every step runs in FP64 whatever the factor's precision (the Gram matrix
// squares the conditioning of A_np).
#pragma once

#include <cfloat>

#include "cpqr_cluster.cuh"

namespace spand {

template <typename T>
struct InterpTask {
  T* Rp;               // p's block row (leading dimension ldp)
  const int32_t* tcol; // m: column of A_pn's j-th column in p's row
  double* G;           // np x np: the Gram matrix; after the factorization T_cf, row-major (r x nf, ld nf)
  double* Rw;          // np x np: row k of R (pivot k) at Rw[k np + j], j = p's dof
  double* P;           // np x np: A_pp[perm, perm], then C_cf (rows < r, cols >= r) and C_ff (both >= r)
  T* cp;               // copy of the coupling blocks before the gather: np x m, then m x np
  int32_t* perm;       // np: c in pivot order, then f in increasing order
  int32_t* rank;       // r
  T* F;                // [C_ff | C_fc], nf x np, leading dimension ldf (factor storage)
  T* XT;               // T_cf, r x nf, leading dimension r (factor storage)
  int32_t p, np, ldp, m, nbeg, nend;  // neighbours: nbrs[nbeg .. nend)
  int32_t r, nf, ldf, pad;            // set once the rank is known
};

// G = A_np^T A_np: one 32 x 32 tile (ti <= tj) per CTA; tile lists are
// (task, ti, tj).  Thread (ty, tx) computes rows 4 ty .. 4 ty + 3 of column
// tx; K = the m coupling columns in chunks of 32.  The tile and its mirror
// image are both stored.
struct InterpTile {
  int32_t task, i0, j0;
};

template <typename T>
__global__ void __launch_bounds__(256) k_interp_gram(const InterpTask<T>* __restrict__ tasks,
                                                     const InterpTile* __restrict__ tiles) {
  const InterpTile tl = tiles[blockIdx.x];
  const InterpTask<T>& d = tasks[tl.task];
  const int r0 = tl.i0, c0 = tl.j0;
  __shared__ double a[32][33], b[32][33];
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int k0 = 0; k0 < d.m; k0 += 32) {
    for (int e = tid; e < 1024; e += 256) {
      const int i = e & 31, kk = e >> 5, k = k0 + kk;
      const T* col = (k < d.m) ? d.Rp + (size_t)d.tcol[k] * d.ldp : nullptr;
      a[i][kk] = (col && r0 + i < d.np) ? (double)col[r0 + i] : 0.0;
      b[kk][i] = (col && c0 + i < d.np) ? (double)col[c0 + i] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      const double bv = b[kk][tx];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = fma(a[4 * ty + q][kk], bv, acc[q]);
    }
    __syncthreads();
  }
  const int c = c0 + tx;
  if (c < d.np)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = r0 + 4 * ty + q;
      if (i < d.np) {
        d.G[i + (size_t)c * d.np] = acc[q];
        d.G[c + (size_t)i * d.np] = acc[q];
      }
    }
}

// Steps 1-2, one task per CTA.  Left-looking pivoted Cholesky: at step k the
// pivot is the largest remaining diagonal (lowest index on ties), and only
// row k of R is formed, R_kj = (G_{pk,j} - sum_{a<k} R_{a,pk} R_{aj}) / R_kk,
// with the remaining diagonals downdated by R_kj^2.  Then f, the rank, and
// T_cf = R_11^{-1} R_12 by back substitution (one column of f per thread),
// row-major into G's storage.  Shared memory: np doubles + np ints.
template <typename T>
__global__ void __launch_bounds__(256) k_interp_factor(const InterpTask<T>* __restrict__ tasks, double eps) {
  const InterpTask<T> d = tasks[blockIdx.x];
  const int np = d.np, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  extern __shared__ __align__(16) unsigned char ip_smem[];
  double* dg = reinterpret_cast<double*>(ip_smem);  // remaining diagonals
  int* used = reinterpret_cast<int*>(dg + np);
  __shared__ double wv[8];
  __shared__ int wj[8];
  __shared__ int piv_sh, stop_sh;
  __shared__ double d0_sh;
  const double* G = d.G;
  double* Rw = d.Rw;
  if (d.m == 0) {  // no coupling: nothing to interpolate, every dof is kept
    for (int i = tid; i < np; i += 256) d.perm[i] = i;
    if (tid == 0) d.rank[0] = np;
    return;
  }
  for (int i = tid; i < np; i += 256) {
    dg[i] = G[i + (size_t)i * np];
    used[i] = 0;
  }
  __syncthreads();
  const int kmax = min(np, d.m);
  int r = kmax;
  for (int k = 0; k < kmax; ++k) {
    double bv = -1.0;
    int bj = INT_MAX;
    for (int i = tid; i < np; i += 256)
      if (!used[i] && (dg[i] > bv || (dg[i] == bv && i < bj))) bv = dg[i], bj = i;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
      if (ov > bv || (ov == bv && oj < bj)) bv = ov, bj = oj;
    }
    if (lane == 0) wv[warp] = bv, wj[warp] = bj;
    __syncthreads();
    if (tid == 0) {
      double v = wv[0];
      int j = wj[0];
      for (int w = 1; w < 8; ++w)
        if (wv[w] > v || (wv[w] == v && wj[w] < j)) v = wv[w], j = wj[w];
      if (k == 0) d0_sh = v;
      // truncation (Sec. 4): stop at the first k with R_kk < eps R_00, i.e.
      // d < eps^2 d_0.  Any positive remainder is kept otherwise, even near
      // the Gram matrix's rounding (about u d_0): keeping a direction never
      // drops anything, while a floor at that level dropped directions the
      // exact (eps = 0) factorization needs.  Only a remainder below u^2 d_0
      // (R_kk below u R_00, where R's row is pure rounding) or a
      // non-positive one ends the factorization early.
      const double floor2 = DBL_EPSILON * DBL_EPSILON;
      stop_sh = (!(v > 0.0) || v < fmax(eps * eps, floor2) * d0_sh) ? 1 : 0;
      piv_sh = j;
      if (!stop_sh) {
        used[j] = 1;
        d.perm[k] = j;
      }
    }
    __syncthreads();
    if (stop_sh) {
      r = k;
      break;
    }
    const int pk = piv_sh;
    const double rkk = sqrt(dg[pk]);
    for (int j = tid; j < np; j += 256) {
      if (used[j]) continue;
      double s = G[j + (size_t)pk * np];
      for (int a = 0; a < k; ++a) s = fma(-Rw[(size_t)a * np + pk], Rw[(size_t)a * np + j], s);
      s /= rkk;
      Rw[(size_t)k * np + j] = s;
      dg[j] -= s * s;
    }
    if (tid == 0) Rw[(size_t)k * np + pk] = rkk;
    __syncthreads();
  }
  if (tid == 0) {
    int o = r;
    for (int i = 0; i < np; ++i)
      if (!used[i]) d.perm[o++] = i;
    d.rank[0] = r;
  }
  __syncthreads();
  // T_cf (r x nf, row-major, ld nf) = R_11^{-1} R_12 into G's storage (G is
  // no longer read)
  const int nf = np - r;
  double* Tt = d.G;
  const int* perm = d.perm;
  for (int jf = tid; jf < nf; jf += 256) {
    const int fj = perm[r + jf];
    for (int a = r - 1; a >= 0; --a) {
      const double* Ra = Rw + (size_t)a * np;
      double s = Ra[fj];
      for (int b = a + 1; b < r; ++b) s = fma(-Ra[perm[b]], Tt[(size_t)b * nf + jf], s);
      Tt[(size_t)a * nf + jf] = s / Ra[perm[a]];
    }
  }
}

// P = A_pp[perm, perm] in FP64 (grid: x = slices, y = task).
template <typename T>
__global__ void __launch_bounds__(256) k_interp_gather_pp(const InterpTask<T>* __restrict__ tasks) {
  const InterpTask<T>& d = tasks[blockIdx.y];
  const int np = d.np;
  const int64_t tot = (int64_t)np * np;
  for (int64_t e = blockIdx.x * 256 + threadIdx.x; e < tot; e += (int64_t)gridDim.x * 256) {
    const int a = (int)(e % np), b = (int)(e / np);
    d.P[e] = (double)d.Rp[d.perm[a] + (size_t)d.perm[b] * d.ldp];
  }
}

// Batched FP64 GEMM, C -= op(A) op(B) (m x n, K = k), 64 x 64 tiles, 256
// threads, 4 x 4 outputs per thread (rows ty + 16 i, columns tx + 16 j).
// op(A): ta = 0, A[i + kk lda]; ta = 1, A[kk + i lda].  op(B): tb = 0,
// B[kk + j ldb]; tb = 1, B[j + kk ldb].
struct DGemmTask {
  const double* A;
  const double* B;
  double* C;
  int32_t lda, ldb, ldc, ta, tb, m, n, k;
};

struct DGemmTile {
  int32_t task, i0, j0;
};

__global__ void __launch_bounds__(256) k_dgemm_sub(const DGemmTask* __restrict__ tasks,
                                                   const DGemmTile* __restrict__ tiles) {
  const DGemmTile tl = tiles[blockIdx.x];
  const DGemmTask g = tasks[tl.task];
  __shared__ double As[16][65], Bs[16][65];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc[4][4] = {};
  for (int k0 = 0; k0 < g.k; k0 += 16) {
    for (int e = tid; e < 1024; e += 256) {
      // A chunk: 64 rows x 16 k; B chunk: 16 k x 64 columns (the index
      // split follows the contiguous direction of each operand)
      const int i = g.ta ? e >> 4 : e & 63, kk = g.ta ? e & 15 : e >> 6;
      const int gi = tl.i0 + i, gk = k0 + kk;
      double v = 0.0;
      if (gi < g.m && gk < g.k) v = g.ta ? g.A[gk + (size_t)gi * g.lda] : g.A[gi + (size_t)gk * g.lda];
      As[kk][i] = v;
      const int j = g.tb ? e & 63 : e >> 4, kb = g.tb ? e >> 6 : e & 15;
      const int gj = tl.j0 + j, gkb = k0 + kb;
      double w = 0.0;
      if (gj < g.n && gkb < g.k) w = g.tb ? g.B[gj + (size_t)gkb * g.ldb] : g.B[gkb + (size_t)gj * g.ldb];
      Bs[kb][j] = w;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      double av[4], bv[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        av[q] = As[kk][ty + 16 * q];
        bv[q] = Bs[kk][tx + 16 * q];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gi = tl.i0 + ty + 16 * i, gj = tl.j0 + tx + 16 * j;
      if (gi < g.m && gj < g.n) g.C[gi + (size_t)gj * g.ldc] -= acc[i][j];
    }
}

// Step 4a: copies of the coupling blocks before the in-place gathers of step
// 4b: p's coupling columns (np x m, column j of A_pn at cp[j np]), then each
// neighbour's block A_qp (w_q x np, column a at w_q a after the previous
// neighbours' blocks).  Grid (CTAs per task, tasks): the warps of a task's
// CTAs take columns, the lanes rows.
template <typename T>
__global__ void __launch_bounds__(256) k_interp_copy(const InterpTask<T>* __restrict__ tasks,
                                                     const CpqrNbr<T>* __restrict__ nbrs,
                                                     const int32_t* __restrict__ cur_size) {
  const InterpTask<T> d = tasks[blockIdx.y];
  const int np = d.np, m = d.m, lane = threadIdx.x & 31;
  const int gw = blockIdx.x * 8 + (threadIdx.x >> 5), nw = gridDim.x * 8;
  for (int j = gw; j < m; j += nw) {
    const T* src = d.Rp + (size_t)d.tcol[j] * d.ldp;
    T* dst = d.cp + (size_t)j * np;
    for (int i = lane; i < np; i += 32) dst[i] = src[i];
  }
  T* cpq = d.cp + (size_t)np * m;
  for (int e = d.nbeg; e < d.nend; ++e) {
    const CpqrNbr<T> nb = nbrs[e];
    const int w = cur_size[nb.q];
    for (int a = gw; a < np; a += nw) {
      const T* src = nb.Rq + (size_t)(nb.off_qp + a) * nb.ldq;
      T* dst = cpq + (size_t)a * w;
      for (int jj = lane; jj < w; jj += 32) dst[jj] = src[jj];
    }
    cpq += (size_t)w * np;
  }
}

// Step 4b, grid (CTAs per task, tasks), after k_interp_copy: the factor
// blocks F = [C_ff | C_fc] (from P, rounded to the factor's type) and
// X^T = T_cf (r x nf, ld r) of the apply's T_p; p keeps A_cc (P's leading
// r x r block), the rows c (pivot order) of its coupling blocks, and every
// neighbour q the columns c of its block A_qp, all gathered from the copies;
// the size of p becomes r (no other task of the colour reads it: the
// interfaces of one colour are not adjacent).
template <typename T>
__global__ void __launch_bounds__(256) k_interp_store(const InterpTask<T>* __restrict__ tasks,
                                                      const CpqrNbr<T>* __restrict__ nbrs,
                                                      int32_t* __restrict__ cur_size) {
  const InterpTask<T> d = tasks[blockIdx.y];
  const int np = d.np, r = d.r, nf = d.nf, m = d.m, lane = threadIdx.x & 31;
  const int gw = blockIdx.x * 8 + (threadIdx.x >> 5), nw = gridDim.x * 8;
  const double* P = d.P;
  for (int b = gw; b < r; b += nw)  // A_cc
    for (int a = lane; a < r; a += 32) d.Rp[a + (size_t)b * d.ldp] = (T)P[a + (size_t)b * np];
  for (int j = gw; j < np; j += nw)  // [C_ff | C_fc]
    for (int i = lane; i < nf; i += 32) {
      const double v = j < nf ? P[(r + i) + (size_t)(r + j) * np] : P[(j - nf) + (size_t)(r + i) * np];
      d.F[i + (size_t)j * d.ldf] = (T)v;
    }
  for (int j = gw; j < nf; j += nw)  // T_cf, column-major ld r
    for (int a = lane; a < r; a += 32) d.XT[a + (size_t)j * r] = (T)d.G[(size_t)a * nf + j];
  for (int j = gw; j < m; j += nw) {  // rows c of p's coupling blocks
    T* dst = d.Rp + (size_t)d.tcol[j] * d.ldp;
    const T* src = d.cp + (size_t)j * np;
    for (int a = lane; a < r; a += 32) dst[a] = src[d.perm[a]];
  }
  const T* cpq = d.cp + (size_t)np * m;
  for (int e = d.nbeg; e < d.nend; ++e) {  // columns c of the neighbours' blocks
    const CpqrNbr<T> nb = nbrs[e];
    const int w = cur_size[nb.q];
    for (int a = gw; a < r; a += nw) {
      T* dst = nb.Rq + (size_t)(nb.off_qp + a) * nb.ldq;
      const T* src = cpq + (size_t)d.perm[a] * w;
      for (int jj = lane; jj < w; jj += 32) dst[jj] = src[jj];
    }
    cpq += (size_t)w * np;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) cur_size[d.p] = r;
}

}  // namespace spand

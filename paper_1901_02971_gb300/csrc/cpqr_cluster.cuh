// Orthogonal sparsification of scaled interfaces (Sec. 2.6.1) on thread-block
// clusters.
//
// For an interface p with |p| = np rows and the coupling A_pn (np x m, all
// current neighbour columns in neighbour order), Householder QR with column
// pivoting (largest remaining column norm; lowest column index on ties) runs
// until the first k with |R_kk| < eps |R_00| (truncation rule of Sec. 4); the
// kept rows W_cn = Q_pc^T A_pn are written back into p's block row and their
// transposes into the neighbours' rows, A_cc = I, and the explicit coarse
// basis Q_pc = H_0 ... H_{r-1} [I_r; 0] is formed.
//
// GB300 mapping: one cluster of C CTAs (C = 1..16) per interface.  The m
// columns are split into C contiguous chunks; each CTA keeps its chunk
// row-major (element (i, j) at chunk[i*ldc + j]) in shared memory when it fits,
// otherwise in global scratch, and updates it with one thread per column.
// Columns are never swapped: the pivot column is retired in place, so after r
// steps the top r rows of every column are W_cn in the original column order.
// Per reflector step the CTAs exchange their pivot candidates and the
// Householder vector through distributed shared memory, with two cluster
// barriers (no spin-waits on global flags).
#pragma once

#include <cooperative_groups.h>

#include "dense_tiles.cuh"

namespace spand {

namespace cg = cooperative_groups;

constexpr int CQ_NT = 256;

template <typename T>
struct CpqrNbr {      // neighbour q of p (Sec. 2.6.1: A_pn spans all of them)
  T* Rq;              // q's block row
  int32_t q, off_pq, off_qp, ldq;
};

template <typename T>
struct CpqrTask {
  T* Rp;              // p's block row (leading dimension ldp)
  T* gwork;           // global fallback for the chunks: C * np * cols_per
  T* V;               // np x np capacity, column k = v_k (v_k[k] = 1, zero above)
  T* tau;             // np
  T* Qc;              // np x np capacity; first r columns = Q_pc on exit
  int32_t p, np, ldp, nbeg, nend, m_max;
};

template <typename T>
struct CqShared {     // fixed part of the dynamic shared memory
  T cand_v[16];       // pivot candidate of every CTA of the cluster (pushed by its owner)
  int cand_j[16];
  T alpha, beta, tau;  // reflector of the current step (pushed by the pivot's owner)
};

// one barrier for the whole cluster (a plain block barrier when C == 1)
__device__ __forceinline__ void cq_sync(cg::cluster_group& cl, int C) {
  if (C == 1) __syncthreads();
  else cl.sync();
}

// dynamic shared memory layout:
//   [CqShared][cstart: (nnb+1) ints][vbuf: np T][norms: cols_per T][chunk: np * ldc T (if resident)]
// `norms` holds the squared trailing norms of the CTA's columns (-1 once the
// column has been a pivot).  Per reflector step k:
//   1. every CTA finds its best column (largest norm, lowest index on ties)
//      and pushes it into every CTA's candidate slots; barrier;
//   2. every thread reduces the C candidates: pivot j*, |R_kk| = sqrt(norm j*)
//      (norms are recomputed exactly, so this is the 2-norm of the pivot's
//      trailing column); the truncation rule is checked here, uniformly;
//   3. the owner of j* forms the reflector (beta = -sign(alpha) |R_kk|,
//      tau = (beta - alpha) / beta, v = x / (alpha - beta)) and pushes alpha,
//      beta, tau and v into every CTA; it retires the column; barrier;
//   4. every CTA applies H_k to its live columns and refreshes their norms.
template <typename T>
__global__ void __launch_bounds__(CQ_NT) k_cpqr_cluster(const CpqrTask<T>* __restrict__ tasks,
                                                       const int32_t* __restrict__ list,
                                                       const CpqrNbr<T>* __restrict__ nbrs,
                                                       int32_t* __restrict__ cur_size, T eps,
                                                       int32_t chunk_smem_bytes) {
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const CpqrTask<T> d = tasks[list[blockIdx.x / C]];
  const int np = d.np;
  const int nnb = d.nend - d.nbeg;
  extern __shared__ __align__(16) unsigned char smraw[];
  CqShared<T>& sh = *reinterpret_cast<CqShared<T>*>(smraw);
  size_t off = (sizeof(CqShared<T>) + 15) & ~size_t(15);
  int* cstart = reinterpret_cast<int*>(smraw + off);
  off += ((size_t)(nnb + 1) * sizeof(int) + 15) & ~size_t(15);
  T* vbuf = reinterpret_cast<T*>(smraw + off);
  off += ((size_t)np * sizeof(T) + 15) & ~size_t(15);
  T* snorm = reinterpret_cast<T*>(smraw + off);
  const size_t norm_off = off;
  __shared__ T red_v[CQ_NT / 32];
  __shared__ int red_j[CQ_NT / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

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
  if (m == 0) {  // every neighbour reduced to nothing: p is kept as it is
    if (rank == 0) {
      for (int64_t x = tid; x < (int64_t)np * np; x += CQ_NT) {
        const int i = (int)(x % np), j = (int)(x / np);
        d.Qc[i + (size_t)j * np] = (i == j) ? T(1) : T(0);
      }
      if (tid == 0) cur_size[d.p] = np;
    }
    return;  // uniform across the cluster (m is the same for every CTA)
  }
  const int cols_per = (m + C - 1) / C;
  const int j0 = min(m, rank * cols_per);
  const int nc = min(m, j0 + cols_per) - j0;
  const int ldc = max(cols_per, 1);
  T* schunk = reinterpret_cast<T*>(smraw + norm_off + (((size_t)ldc * sizeof(T) + 15) & ~size_t(15)));
  const bool resident = (int64_t)np * ldc * (int64_t)sizeof(T) <= (int64_t)chunk_smem_bytes;
  T* chunk = resident ? schunk : d.gwork + (size_t)rank * np * ldc;

  // neighbour of a global column: largest e with cstart[e] <= j
  auto owner_nbr = [&](int j) {
    int lo = 0, hi = nnb - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (cstart[mid] <= j) lo = mid; else hi = mid - 1;
    }
    return lo;
  };

  // ---- gather my columns of A_pn and their norms
  for (int jl = warp; jl < nc; jl += CQ_NT / 32) {
    const int j = j0 + jl;
    const int e = owner_nbr(j);
    const CpqrNbr<T> nb = nbrs[d.nbeg + e];
    const T* src = d.Rp + (size_t)(nb.off_pq + (j - cstart[e])) * d.ldp;
    T s = 0;
    for (int i = lane; i < np; i += 32) {
      const T v = src[i];
      chunk[(size_t)i * ldc + jl] = v;
      s += v * v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) snorm[jl] = s;
  }
  __syncthreads();

  const int kmax = min(np, m);
  int r = kmax;
  T r00 = T(0);
  for (int k = 0; k < kmax; ++k) {
    // 1. local pivot candidate
    T bv = T(-1);
    int bj = INT_MAX;
    for (int jl = tid; jl < nc; jl += CQ_NT) {
      const T v = snorm[jl];
      if (v > bv) { bv = v; bj = j0 + jl; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
      if (ov > bv || (ov == bv && oj < bj)) { bv = ov; bj = oj; }
    }
    if (lane == 0) { red_v[warp] = bv; red_j[warp] = bj; }
    __syncthreads();
    bv = red_v[0];
    bj = red_j[0];
    for (int w = 1; w < CQ_NT / 32; ++w)
      if (red_v[w] > bv || (red_v[w] == bv && red_j[w] < bj)) { bv = red_v[w]; bj = red_j[w]; }
    T gv = bv;
    int gj = bj;
    if (C > 1) {
      if (tid < C) {  // push my candidate into slot `rank` of CTA `tid`
        CqShared<T>* o = cluster.map_shared_rank(&sh, tid);
        o->cand_v[rank] = bv;
        o->cand_j[rank] = bj;
      }
      cluster.sync();
      gv = T(-1);
      gj = INT_MAX;
      for (int q = 0; q < C; ++q) {
        const T v = sh.cand_v[q];
        const int j = sh.cand_j[q];
        if (v > gv || (v == gv && j < gj)) { gv = v; gj = j; }
      }
    }
    if (gj == INT_MAX) gj = 0;  // unreachable: k < kmax <= m leaves a column
    // 2. |R_kk| and the truncation rule (same values in every thread)
    const T rkk = sqrt(gv > T(0) ? gv : T(0));
    if (k == 0) r00 = rkk;
    if (r00 == T(0) || rkk < eps * r00) {
      r = k;
      break;
    }
    const int owner = min(C - 1, gj / max(cols_per, 1));
    // 3. the owner forms the reflector and pushes it to every CTA
    if (rank == owner) {
      const int jl = gj - j0;
      const T alpha = chunk[(size_t)k * ldc + jl];
      T beta, tau, scal;
      if (rkk == T(0)) {
        beta = T(0);
        tau = T(0);
        scal = T(0);
      } else {
        beta = alpha >= T(0) ? -rkk : rkk;
        tau = (beta - alpha) / beta;
        scal = T(1) / (alpha - beta);
      }
      for (int i = k + tid; i < np; i += CQ_NT) {
        const T v = (i == k) ? T(1) : chunk[(size_t)i * ldc + jl] * scal;
        for (int q = 0; q < C; ++q) cluster.map_shared_rank(vbuf, q)[i] = v;
        d.V[i + (size_t)k * np] = v;
      }
      for (int i = tid; i < k; i += CQ_NT) d.V[i + (size_t)k * np] = T(0);
      if (tid < C) {
        CqShared<T>* o = cluster.map_shared_rank(&sh, tid);
        o->alpha = alpha;
        o->beta = beta;
        o->tau = tau;
      }
      if (tid == 0) d.tau[k] = tau;
    }
    cq_sync(cluster, C);
    const T tau = sh.tau;
    if (rank == owner) {  // retire the pivot column: R_kk = beta, zeros below
      const int jl = gj - j0;
      for (int i = k + tid; i < np; i += CQ_NT) chunk[(size_t)i * ldc + jl] = (i == k) ? sh.beta : T(0);
      if (tid == 0) snorm[jl] = T(-1);
    }
    // 4. apply H_k to my live columns, refresh their trailing norms
    for (int jl = tid; jl < nc; jl += CQ_NT) {
      if (jl == gj - j0) continue;
      if (snorm[jl] < T(0)) continue;
      T* __restrict__ col = chunk + jl;    // disjoint from vbuf: lets the loads run ahead of the stores
      const T* __restrict__ vb = vbuf;
      // w = v^T col[k:], four independent partial sums
      T w0 = 0, w1 = 0, w2 = 0, w3 = 0;
      int i = k;
      for (; i + 4 <= np; i += 4) {
        w0 += vb[i] * col[(size_t)i * ldc];
        w1 += vb[i + 1] * col[(size_t)(i + 1) * ldc];
        w2 += vb[i + 2] * col[(size_t)(i + 2) * ldc];
        w3 += vb[i + 3] * col[(size_t)(i + 3) * ldc];
      }
      for (; i < np; ++i) w0 += vb[i] * col[(size_t)i * ldc];
      const T w = ((w0 + w1) + (w2 + w3)) * tau;
      col[(size_t)k * ldc] -= w;  // v_k = 1
      // update rows k+1.. and their squared norm
      T q0 = 0, q1 = 0, q2 = 0, q3 = 0;
      i = k + 1;
      for (; i + 4 <= np; i += 4) {
        const T x0 = col[(size_t)i * ldc] - w * vb[i];
        const T x1 = col[(size_t)(i + 1) * ldc] - w * vb[i + 1];
        const T x2 = col[(size_t)(i + 2) * ldc] - w * vb[i + 2];
        const T x3 = col[(size_t)(i + 3) * ldc] - w * vb[i + 3];
        col[(size_t)i * ldc] = x0;
        col[(size_t)(i + 1) * ldc] = x1;
        col[(size_t)(i + 2) * ldc] = x2;
        col[(size_t)(i + 3) * ldc] = x3;
        q0 += x0 * x0;
        q1 += x1 * x1;
        q2 += x2 * x2;
        q3 += x3 * x3;
      }
      for (; i < np; ++i) {
        const T x = col[(size_t)i * ldc] - w * vb[i];
        col[(size_t)i * ldc] = x;
        q0 += x * x;
      }
      snorm[jl] = (q0 + q1) + (q2 + q3);
    }
    __syncthreads();
  }
  // Rows 0..r-1 of every column now hold W_cn in the original column order
  // (the pivot found at step r, if any, was not touched).
  // ---- write back W_cn into p's row and the transposes into the neighbours
  for (int64_t x = tid; x < (int64_t)r * nc; x += CQ_NT) {
    const int i = (int)(x % r), jl = (int)(x / r);
    const int j = j0 + jl;
    const int e = owner_nbr(j);
    const CpqrNbr<T> nb = nbrs[d.nbeg + e];
    const int cc = j - cstart[e];
    const T val = chunk[(size_t)i * ldc + jl];
    d.Rp[i + (size_t)(nb.off_pq + cc) * d.ldp] = val;
    nb.Rq[cc + (size_t)(nb.off_qp + i) * nb.ldq] = val;
  }
  if (rank == 0)
    for (int64_t x = tid; x < (int64_t)r * r; x += CQ_NT) {
      const int i = (int)(x % r), j = (int)(x / r);
      d.Rp[i + (size_t)j * d.ldp] = (i == j) ? T(1) : T(0);
    }
  if (C > 1) cluster.sync();  // every V column and tau is visible cluster-wide
  // ---- Q_pc e_c = H_0 ... H_c e_c (H_k e_c = e_c for k > c), one warp per
  // column, the column held in registers (lane l owns rows l, l+32, ...)
  constexpr int QR = 16;  // rows per lane held in registers
  if (np > 32 * QR) {     // tall interfaces: the column lives in global memory
    for (int c = rank * (CQ_NT / 32) + warp; c < r; c += C * (CQ_NT / 32)) {
      T* col = d.Qc + (size_t)c * np;
      for (int i = lane; i < np; i += 32) col[i] = (i == c) ? T(1) : T(0);
      __syncwarp();
      for (int k = c; k >= 0; --k) {
        const T tk = d.tau[k];
        if (tk == T(0)) continue;
        const T* v = d.V + (size_t)k * np;
        T w = 0;
        for (int i = k + lane; i < np; i += 32) w += v[i] * col[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        w *= tk;
        for (int i = k + lane; i < np; i += 32) col[i] -= w * v[i];
        __syncwarp();
      }
    }
  }
  for (int c = rank * (CQ_NT / 32) + warp; np <= 32 * QR && c < r; c += C * (CQ_NT / 32)) {
    T col[QR];
#pragma unroll
    for (int q = 0; q < QR; ++q) col[q] = (lane + 32 * q == c) ? T(1) : T(0);
    for (int k = c; k >= 0; --k) {
      const T tk = d.tau[k];
      if (tk == T(0)) continue;
      const T* v = d.V + (size_t)k * np;
      T w = 0;
#pragma unroll
      for (int q = 0; q < QR; ++q) {
        const int i = lane + 32 * q;
        if (i >= k && i < np) w += v[i] * col[q];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
      w *= tk;
#pragma unroll
      for (int q = 0; q < QR; ++q) {
        const int i = lane + 32 * q;
        if (i >= k && i < np) col[q] -= w * v[i];
      }
    }
    T* out = d.Qc + (size_t)c * np;
#pragma unroll
    for (int q = 0; q < QR; ++q) {
      const int i = lane + 32 * q;
      if (i < np) out[i] = col[q];
    }
  }
  if (rank == 0 && tid == 0) cur_size[d.p] = r;
  if (C > 1) cluster.sync();  // no CTA leaves while others may still write into its shared memory
}

}  // namespace spand

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
  T* norms;           // m_max: squared trailing column norms, -1 once pivoted
  T* V;               // np x np capacity, column k = v_k (v_k[k] = 1, zero above)
  T* tau;             // np
  T* Qc;              // np x np capacity; first r columns = Q_pc on exit
  int32_t p, np, ldp, nbeg, nend, m_max;
};

template <typename T>
struct CqShared {     // fixed part of the dynamic shared memory
  T cand_v;
  int cand_j;
  T beta, tau;
  int stop;
};

// dynamic shared memory layout:
//   [CqShared][cstart: (nnb+1) ints][vbuf: np T][chunk: np * ldc T (if resident)]
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
  T* schunk = reinterpret_cast<T*>(smraw + off);
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
    if (lane == 0) d.norms[j] = s;
  }
  __syncthreads();

  const int kmax = min(np, m);
  int r = kmax;
  T r00 = T(0);
  for (int k = 0; k < kmax; ++k) {
    // (a) local pivot candidate: largest norm, lowest global column on ties
    T bv = T(-1);
    int bj = INT_MAX;
    for (int jl = tid; jl < nc; jl += CQ_NT) {
      const T v = d.norms[j0 + jl];
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
    if (tid == 0) {
      for (int w = 1; w < CQ_NT / 32; ++w)
        if (red_v[w] > bv || (red_v[w] == bv && red_j[w] < bj)) { bv = red_v[w]; bj = red_j[w]; }
      sh.cand_v = bv;
      sh.cand_j = bj;
    }
    cluster.sync();
    // every CTA reduces the C candidates in the same order -> same pivot
    T gv = T(-1);
    int gj = INT_MAX;
    for (int q = 0; q < C; ++q) {
      const CqShared<T>* o = cluster.map_shared_rank(&sh, q);
      const T v = o->cand_v;
      const int j = o->cand_j;
      if (v > gv || (v == gv && j < gj)) { gv = v; gj = j; }
    }
    if (gj == INT_MAX) gj = 0;  // unreachable: k < kmax <= m leaves a column
    const int owner = min(C - 1, gj / max(cols_per, 1));
    // (b) the owner forms the Householder reflector of its pivot column
    if (rank == owner) {
      const int jl = gj - j0;
      T s = 0;
      for (int i = k + 1 + tid; i < np; i += CQ_NT) {
        const T x = chunk[(size_t)i * ldc + jl];
        s += x * x;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      __syncthreads();
      if (lane == 0) red_v[warp] = s;
      __syncthreads();
      if (tid == 0) {
        T sig = 0;
        for (int w = 0; w < CQ_NT / 32; ++w) sig += red_v[w];
        const T alpha = chunk[(size_t)k * ldc + jl];
        T beta, tau;
        if (sig == T(0)) {
          beta = alpha;
          tau = T(0);
        } else {
          const T nrm = sqrt(alpha * alpha + sig);
          beta = alpha >= T(0) ? -nrm : nrm;
          tau = (beta - alpha) / beta;
        }
        sh.beta = beta;
        sh.tau = tau;
        vbuf[k] = T(1);
        d.norms[gj] = T(-1);
        d.tau[k] = tau;
      }
      __syncthreads();
      const T alpha = chunk[(size_t)k * ldc + jl];
      const T beta = sh.beta, tau = sh.tau;
      const T scal = (tau == T(0)) ? T(0) : T(1) / (alpha - beta);
      for (int i = k + 1 + tid; i < np; i += CQ_NT) {
        const T v = chunk[(size_t)i * ldc + jl] * scal;
        vbuf[i] = v;
        chunk[(size_t)i * ldc + jl] = T(0);
      }
      __syncthreads();  // vbuf entries come from other threads
      for (int i = tid; i < np; i += CQ_NT) d.V[i + (size_t)k * np] = i < k ? T(0) : (i == k ? T(1) : vbuf[i]);
      __syncthreads();
      if (tid == 0) chunk[(size_t)k * ldc + jl] = beta;
    }
    cluster.sync();
    // (c) everyone takes the reflector from the owner and checks the rule
    const CqShared<T>* osh = cluster.map_shared_rank(&sh, owner);
    const T beta = osh->beta, tau = osh->tau;
    const T rkk = fabs(beta);
    if (k == 0) r00 = rkk;
    if (r00 == T(0) || rkk < eps * r00) {
      r = k;
      break;  // uniform: every CTA read the same beta
    }
    if (rank != owner) {
      const T* ov = cluster.map_shared_rank(vbuf, owner);
      for (int i = k + tid; i < np; i += CQ_NT) vbuf[i] = ov[i];
    }
    __syncthreads();
    // (d) apply H_k to my remaining columns, refresh their trailing norms
    for (int jl = tid; jl < nc; jl += CQ_NT) {
      if (d.norms[j0 + jl] < T(0)) continue;
      T w = 0;
      for (int i = k; i < np; ++i) w += vbuf[i] * chunk[(size_t)i * ldc + jl];
      w *= tau;
      T s = 0;
      for (int i = k; i < np; ++i) {
        const T x = chunk[(size_t)i * ldc + jl] - w * vbuf[i];
        chunk[(size_t)i * ldc + jl] = x;
        if (i > k) s += x * x;
      }
      d.norms[j0 + jl] = s;
    }
    __syncthreads();
  }
  // the owner of step r may have retired a column that is not kept: its top r
  // rows are untouched, so every column's rows 0..r-1 hold W_cn.
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
  // ---- Q_pc e_c = H_0 ... H_c e_c (H_k e_c = e_c for k > c), one warp per column
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
  if (rank == 0 && tid == 0) cur_size[d.p] = r;
  cluster.sync();  // keep every CTA's shared memory alive until all DSMEM reads are done
}

}  // namespace spand

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
// column-major (column jl at chunk[jl * L], L = cq_ld(np) >= np rows) in
// shared memory when it fits, otherwise in global scratch.  One thread owns a
// column (CQ_CPT at most) and streams it with 16-byte vector loads; the stride L
// is chosen so that the 8 threads of a quarter-warp hit distinct bank groups.
// Columns are never swapped: the pivot column is retired in place, so after r
// steps the top r rows of every column are W_cn in the original column order.
// Per reflector step the CTAs exchange warp pivot candidates and the
// Householder vector through distributed shared memory, with two cluster
// barriers and no spin-waits.
#pragma once

#include <cooperative_groups.h>

#include "dense_tiles.cuh"

namespace spand {

namespace cg = cooperative_groups;

constexpr int CQ_NT = 256;          // threads per CTA
constexpr int CQ_NW = CQ_NT / 32;   // warps per CTA
constexpr int CQ_MAXC = 16;         // largest cluster
constexpr int CQ_CPT = 4;           // columns per thread at most (the host sizes clusters for it)

template <typename T>
struct CpqrNbr {      // neighbour q of p (Sec. 2.6.1: A_pn spans all of them)
  T* Rq;              // q's block row
  int32_t q, off_pq, off_qp, ldq;
};

template <typename T>
struct CpqrTask {
  T* Rp;              // p's block row (leading dimension ldp)
  T* gwork;           // global chunk storage when it does not fit in shared memory: C * L * cols_per
  T* V;               // np x np capacity, column k = v_k (v_k[k] = 1, rows above k unused)
  T* tau;             // np
  T* Qc;              // np x np capacity; first r columns = Q_pc on exit
  int32_t p, np, ldp, nbeg, nend, m_max;
};

template <typename T>
struct CqVec;
template <>
struct CqVec<float> {
  typedef float4 t;
};
template <>
struct CqVec<double> {
  typedef double2 t;
};

// Column stride of a chunk (elements): the smallest L >= np that is a whole
// number of 16-byte vectors and whose 16-byte stride is odd, so that the
// vector loads of 8 consecutive columns at one row fall into 8 distinct groups
// of 4 banks.
template <typename T>
__host__ __device__ inline int cq_ld(int np) {
  constexpr int vw = 16 / (int)sizeof(T);
  int g = (np + vw - 1) / vw;  // vectors per column
  if (g < 1) g = 1;
  if ((g & 1) == 0) ++g;
  return g * vw;
}

template <typename T>
struct CqShared {     // fixed part of the dynamic shared memory
  T cand_v[CQ_MAXC * CQ_NW];  // warp pivot candidates of the whole cluster (pushed by their owners)
  int cand_j[CQ_MAXC * CQ_NW];
  T tau;                      // reflector of the current step (pushed by the pivot's owner)
};

// Fixed shared memory before the chunk: CqShared, the neighbour column starts
// (nnb + 1 ints) and the broadcast reflector (L elements), each 16-byte aligned.
template <typename T>
__host__ __device__ inline size_t cq_fixed_smem(int nnb, int np) {
  return ((sizeof(CqShared<T>) + 15) & ~size_t(15)) + (((size_t)(nnb + 1) * sizeof(int) + 15) & ~size_t(15)) +
         (((size_t)cq_ld<T>(np) * sizeof(T) + 15) & ~size_t(15));
}

// one barrier for the whole cluster (a plain block barrier when C == 1)
__device__ __forceinline__ void cq_sync(cg::cluster_group& cl, int C) {
  if (C == 1) __syncthreads();
  else cl.sync();
}

// Per reflector step k:
//   1. every warp reduces its threads' best live columns (largest squared
//      trailing norm, lowest index on ties) and pushes the result into slot
//      (rank, warp) of every CTA; barrier;
//   2. every thread reduces the C * 8 candidates: pivot j*, |R_kk| = sqrt(norm)
//      (norms are recomputed exactly each step); the truncation rule is
//      checked here, uniformly;
//   3. the CTA owning j* forms the reflector (beta = -sign(alpha) |R_kk|,
//      tau = (beta - alpha) / beta, v = x / (alpha - beta)), pushes v and tau
//      into every CTA and retires the column (R_kk = beta, zeros below);
//      barrier;
//   4. every thread applies H_k to its live columns and recomputes their
//      trailing norms.
template <typename T, bool RES>
__global__ void __launch_bounds__(CQ_NT) k_cpqr_cluster(const CpqrTask<T>* __restrict__ tasks,
                                                       const int32_t* __restrict__ list,
                                                       const CpqrNbr<T>* __restrict__ nbrs,
                                                       int32_t* __restrict__ cur_size, T eps) {
  typedef typename CqVec<T>::t V;
  constexpr int VW = 16 / (int)sizeof(T);
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const CpqrTask<T> d = tasks[list[blockIdx.x / C]];
  const int np = d.np;
  const int L = cq_ld<T>(np);
  const int ng = (np + VW - 1) / VW;  // vectors per column that hold rows < np
  const int nnb = d.nend - d.nbeg;
  extern __shared__ __align__(16) unsigned char smraw[];
  CqShared<T>& sh = *reinterpret_cast<CqShared<T>*>(smraw);
  size_t off = (sizeof(CqShared<T>) + 15) & ~size_t(15);
  int* cstart = reinterpret_cast<int*>(smraw + off);
  off += ((size_t)(nnb + 1) * sizeof(int) + 15) & ~size_t(15);
  T* vbuf = reinterpret_cast<T*>(smraw + off);
  off += ((size_t)L * sizeof(T) + 15) & ~size_t(15);
  T* schunk = reinterpret_cast<T*>(smraw + off);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  if (tid == 0) {
    int m = 0;
    for (int e = 0; e < nnb; ++e) {
      cstart[e] = m;
      m += cur_size[nbrs[d.nbeg + e].q];
    }
    cstart[nnb] = m;
  }
  for (int i = tid; i < L; i += CQ_NT) vbuf[i] = T(0);
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
  T* __restrict__ chunk = RES ? schunk : d.gwork + (size_t)rank * L * cols_per;

  // neighbour of a global column: largest e with cstart[e] <= j
  auto owner_nbr = [&](int j) {
    int lo = 0, hi = nnb - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (cstart[mid] <= j) lo = mid; else hi = mid - 1;
    }
    return lo;
  };

  // ---- gather my columns of A_pn (one warp per column, coalesced), zero the
  // padding rows of the last vector
  for (int jl = warp; jl < nc; jl += CQ_NW) {
    const int j = j0 + jl;
    const int e = owner_nbr(j);
    const CpqrNbr<T> nb = nbrs[d.nbeg + e];
    const T* src = d.Rp + (size_t)(nb.off_pq + (j - cstart[e])) * d.ldp;
    T* dst = chunk + (size_t)jl * L;
    for (int i = lane; i < ng * VW; i += 32) dst[i] = i < np ? src[i] : T(0);
  }
  __syncthreads();
  // thread t owns local columns t, t + CQ_NT, ...; squared norms (-1: retired or absent)
  T nrm[CQ_CPT];
#pragma unroll
  for (int c = 0; c < CQ_CPT; ++c) {
    const int jl = tid + c * CQ_NT;
    nrm[c] = T(-1);
    if (jl < nc) {
      const V* cv = reinterpret_cast<const V*>(chunk + (size_t)jl * L);
      T s = 0;
      for (int g = 0; g < ng; ++g) {
        const V x = cv[g];
        if constexpr (VW == 4) s += x.x * x.x + x.y * x.y + x.z * x.z + x.w * x.w;
        else s += x.x * x.x + x.y * x.y;
      }
      nrm[c] = s;
    }
  }

  const int kmax = min(np, m);
  int r = kmax;
  T r00 = T(0);
  for (int k = 0; k < kmax; ++k) {
    // 1. warp candidates -> every CTA
    T bv = T(-1);
    int bj = INT_MAX;
#pragma unroll
    for (int c = 0; c < CQ_CPT; ++c)
      if (nrm[c] > bv) {
        bv = nrm[c];
        bj = j0 + tid + c * CQ_NT;
      }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
      if (ov > bv || (ov == bv && oj < bj)) {
        bv = ov;
        bj = oj;
      }
    }
    if (lane < C) {  // lane q pushes this warp's candidate into CTA q
      CqShared<T>* o = C == 1 ? &sh : cluster.map_shared_rank(&sh, lane);
      o->cand_v[rank * CQ_NW + warp] = bv;
      o->cand_j[rank * CQ_NW + warp] = bj;
    }
    cq_sync(cluster, C);
    // 2. pivot and |R_kk| (identical in every thread of the cluster)
    T gv = T(-1);
    int gj = INT_MAX;
    for (int q = lane; q < C * CQ_NW; q += 32) {
      const T v = sh.cand_v[q];
      const int j = sh.cand_j[q];
      if (v > gv || (v == gv && j < gj)) {
        gv = v;
        gj = j;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T ov = __shfl_xor_sync(0xffffffffu, gv, o);
      const int oj = __shfl_xor_sync(0xffffffffu, gj, o);
      if (ov > gv || (ov == gv && oj < gj)) {
        gv = ov;
        gj = oj;
      }
    }
    if (gj == INT_MAX) gj = 0;  // unreachable: k < kmax <= m leaves a live column
    const T rkk = sqrt(gv > T(0) ? gv : T(0));
    if (k == 0) r00 = rkk;
    if (r00 == T(0) || rkk < eps * r00) {
      r = k;
      break;
    }
    const int owner = min(C - 1, gj / cols_per);
#pragma unroll
    for (int c = 0; c < CQ_CPT; ++c)
      if (j0 + tid + c * CQ_NT == gj) nrm[c] = T(-1);  // the pivot column retires
    // 3. the owner forms the reflector, pushes it, retires the pivot column
    if (rank == owner) {
      T* col = chunk + (size_t)(gj - j0) * L;
      const T alpha = col[k];
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
      const int i0 = (k / VW) * VW;
      for (int i = i0 + tid; i < ng * VW; i += CQ_NT) {
        const T x = col[i];
        const T v = i < k ? T(0) : (i == k ? T(1) : x * scal);
        if (C == 1) {
          vbuf[i] = v;
        } else {
          for (int q = 0; q < C; ++q) cluster.map_shared_rank(vbuf, q)[i] = v;
        }
        if (i >= k && i < np) d.V[i + (size_t)k * np] = v;
        if (i >= k) col[i] = (i == k) ? beta : T(0);
      }
      if (tid < C) {
        CqShared<T>* o = C == 1 ? &sh : cluster.map_shared_rank(&sh, tid);
        o->tau = tau;
      }
      if (tid == 0) d.tau[k] = tau;
    }
    cq_sync(cluster, C);
    const T tau = sh.tau;
    // 4. apply H_k to my live columns, recompute their trailing norms
    const int gs = k / VW;
    const V* __restrict__ vv = reinterpret_cast<const V*>(vbuf);
#pragma unroll
    for (int c = 0; c < CQ_CPT; ++c) {
      if (nrm[c] < T(0)) continue;
      V* __restrict__ cv = reinterpret_cast<V*>(chunk + (size_t)(tid + c * CQ_NT) * L);
      T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
#pragma unroll 2
      for (int g = gs; g < ng; ++g) {
        const V x = cv[g], v = vv[g];
        a0 = fma(x.x, v.x, a0);
        a1 = fma(x.y, v.y, a1);
        if constexpr (VW == 4) {
          a2 = fma(x.z, v.z, a2);
          a3 = fma(x.w, v.w, a3);
        }
      }
      const T w = ((a0 + a1) + (a2 + a3)) * tau;
      T q0 = 0, q1 = 0, q2 = 0, q3 = 0;
      {  // first vector: rows <= k do not enter the trailing norm
        V x = cv[gs];
        const V v = vv[gs];
        const int rb = gs * VW;
        x.x = fma(-w, v.x, x.x);
        x.y = fma(-w, v.y, x.y);
        if (rb > k) q0 = x.x * x.x;
        if (rb + 1 > k) q1 = x.y * x.y;
        if constexpr (VW == 4) {
          x.z = fma(-w, v.z, x.z);
          x.w = fma(-w, v.w, x.w);
          if (rb + 2 > k) q2 = x.z * x.z;
          if (rb + 3 > k) q3 = x.w * x.w;
        }
        cv[gs] = x;
      }
#pragma unroll 2
      for (int g = gs + 1; g < ng; ++g) {
        V x = cv[g];
        const V v = vv[g];
        x.x = fma(-w, v.x, x.x);
        x.y = fma(-w, v.y, x.y);
        q0 = fma(x.x, x.x, q0);
        q1 = fma(x.y, x.y, q1);
        if constexpr (VW == 4) {
          x.z = fma(-w, v.z, x.z);
          x.w = fma(-w, v.w, x.w);
          q2 = fma(x.z, x.z, q2);
          q3 = fma(x.w, x.w, q3);
        }
        cv[g] = x;
      }
      nrm[c] = (q0 + q1) + (q2 + q3);
    }
  }
  __syncthreads();
  // Rows 0..r-1 of every column now hold W_cn in the original column order
  // (the pivot found at step r, if any, was not touched).
  // ---- write back W_cn into p's row (one warp per column, coalesced) ...
  for (int jl = warp; jl < nc; jl += CQ_NW) {
    const int j = j0 + jl;
    const int e = owner_nbr(j);
    const CpqrNbr<T> nb = nbrs[d.nbeg + e];
    T* dst = d.Rp + (size_t)(nb.off_pq + (j - cstart[e])) * d.ldp;
    const T* src = chunk + (size_t)jl * L;
    for (int i = lane; i < r; i += 32) dst[i] = src[i];
  }
  // ... and its transpose into the neighbours' rows (one thread per column)
  for (int jl = tid; jl < nc; jl += CQ_NT) {
    const int j = j0 + jl;
    const int e = owner_nbr(j);
    const CpqrNbr<T> nb = nbrs[d.nbeg + e];
    const int cc = j - cstart[e];
    const T* src = chunk + (size_t)jl * L;
    for (int i = 0; i < r; ++i) nb.Rq[cc + (size_t)(nb.off_qp + i) * nb.ldq] = src[i];
  }
  if (rank == 0)
    for (int64_t x = tid; x < (int64_t)r * r; x += CQ_NT) {
      const int i = (int)(x % r), j = (int)(x / r);
      d.Rp[i + (size_t)j * d.ldp] = (i == j) ? T(1) : T(0);
    }
  if (C > 1) cluster.sync();  // every V column and tau is visible cluster-wide
  else __syncthreads();
  // ---- Q_pc e_c = H_0 ... H_c e_c (H_k e_c = e_c for k > c), one warp per
  // column, the column held in registers (lane l owns rows l, l+32, ...).  The
  // reflectors are read from a shared-memory copy of V when it fits in the
  // chunk's space (free again after the write-back).
  const T* Vsrc = d.V;
  if (RES && (size_t)np * r <= (size_t)L * cols_per) {
    T* Vs = schunk;
    for (int64_t x = tid; x < (int64_t)np * r; x += CQ_NT) {
      const int i = (int)(x % np), k = (int)(x / np);
      Vs[x] = i >= k ? __ldcg(d.V + i + (size_t)k * np) : T(0);  // written by other CTAs: read through L2
    }
    __syncthreads();
    Vsrc = Vs;
  }
  constexpr int QR = 16;  // rows per lane held in registers
  if (np > 32 * QR) {     // tall interfaces: the column lives in global memory
    for (int c = rank * CQ_NW + warp; c < r; c += C * CQ_NW) {
      T* col = d.Qc + (size_t)c * np;
      for (int i = lane; i < np; i += 32) col[i] = (i == c) ? T(1) : T(0);
      __syncwarp();
      for (int k = c; k >= 0; --k) {
        const T tk = __ldcg(d.tau + k);
        if (tk == T(0)) continue;
        const T* v = Vsrc + (size_t)k * np;
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
  for (int c = rank * CQ_NW + warp; np <= 32 * QR && c < r; c += C * CQ_NW) {
    T col[QR];
#pragma unroll
    for (int q = 0; q < QR; ++q) col[q] = (lane + 32 * q == c) ? T(1) : T(0);
    for (int k = c; k >= 0; --k) {
      const T tk = __ldcg(d.tau + k);
      if (tk == T(0)) continue;
      const T* v = Vsrc + (size_t)k * np;
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

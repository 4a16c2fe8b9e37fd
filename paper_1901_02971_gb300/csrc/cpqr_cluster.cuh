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
  T* tau;             // np (unused: every CTA keeps the taus in shared memory)
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
  // warp pivot candidates of the whole cluster (pushed by their owners),
  // double-buffered by step parity: with one barrier per step, a fast warp
  // pushes step k+1 while a slow one may still read step k
  T cand_v[2][CQ_MAXC * CQ_NW];
  int cand_j[2][CQ_MAXC * CQ_NW];
};

__host__ __device__ inline size_t cq_al16(size_t b) { return (b + 15) & ~size_t(15); }

// Fixed shared memory before the chunk, each part 16-byte aligned: CqShared,
// the neighbour descriptors (nnb), their column starts (nnb + 1 ints), the
// pivot column copy (L elements), the tau of every reflector (np) and, per
// local column, its neighbour and its column in p's block row (2 cols_per ints).
template <typename T>
__host__ __device__ inline size_t cq_fixed_smem(int nnb, int np, int cols_per) {
  return cq_al16(sizeof(CqShared<T>)) + cq_al16((size_t)nnb * sizeof(CpqrNbr<T>)) +
         cq_al16((size_t)(nnb + 1) * sizeof(int)) + cq_al16((size_t)cq_ld<T>(np) * sizeof(T)) +
         cq_al16((size_t)(np > 0 ? np : 1) * sizeof(T)) + cq_al16((size_t)2 * (cols_per > 0 ? cols_per : 1) * sizeof(int));
}

// Warp-wide (largest value, lowest index on ties); every lane gets the result.
// Values are squared norms (>= 0) or -1 for absent/retired columns.
__device__ __forceinline__ void cq_warp_argmax(float& v, int& j) {
  // for floats >= 0 the signed-integer order of the bit patterns is the float
  // order, and every negative float is a negative integer
  const int best = __reduce_max_sync(0xffffffffu, __float_as_int(v));
  const int jj = __reduce_min_sync(0xffffffffu, __float_as_int(v) == best ? j : INT_MAX);
  v = __int_as_float(best);
  j = jj;
}
__device__ __forceinline__ void cq_warp_argmax(double& v, int& j) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int oj = __shfl_xor_sync(0xffffffffu, j, o);
    if (ov > v || (ov == v && oj < j)) {
      v = ov;
      j = oj;
    }
  }
}

// one barrier for the whole cluster (a plain block barrier when C == 1)
__device__ __forceinline__ void cq_sync(cg::cluster_group& cl, int C) {
  if (C == 1) __syncthreads();
  else cl.sync();
}

// Q_pc e_c = H_0 ... H_c e_c (H_k e_c = e_c for k > c) for the columns c of
// this warp (one warp per column over the whole cluster), the column held in
// registers: lane l owns rows l + 32 q, q < QR (np <= 32 QR).
template <typename T, int QR>
__device__ __forceinline__ void cq_form_q(const CpqrTask<T>& d, const T* Vsrc, const T* tau_s, int r, int np,
                                          int rank, int C) {
  // two columns per warp, their reflector chains interleaved (independent
  // shuffle reductions); c1 > c0, so H_k for c0 < k <= c1 touches c1 only
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = C * CQ_NW, w0 = rank * CQ_NW + warp;
  for (int c0 = w0; c0 < r; c0 += 2 * nwarps) {
    const int c1 = c0 + nwarps;  // may be >= r (then only c0 is formed)
    const bool two = c1 < r;
    T a[QR], b[QR];
#pragma unroll
    for (int q = 0; q < QR; ++q) {
      a[q] = (lane + 32 * q == c0) ? T(1) : T(0);
      b[q] = (lane + 32 * q == c1) ? T(1) : T(0);
    }
    for (int k = two ? c1 : c0; k >= 0; --k) {
      const T tk = tau_s[k];
      if (tk == T(0)) continue;
      const bool doa = k <= c0;
      const T* v = Vsrc + (size_t)k * np;
      T vr[QR];
      T wa = 0, wb = 0;
#pragma unroll
      for (int q = 0; q < QR; ++q) {
        const int i = lane + 32 * q;
        vr[q] = (i >= k && i < np) ? v[i] : T(0);
        wa = fma(vr[q], a[q], wa);
        wb = fma(vr[q], b[q], wb);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        wa += __shfl_xor_sync(0xffffffffu, wa, o);
        wb += __shfl_xor_sync(0xffffffffu, wb, o);
      }
      wa = doa ? wa * tk : T(0);
      wb *= tk;
#pragma unroll
      for (int q = 0; q < QR; ++q) {
        a[q] = fma(-wa, vr[q], a[q]);
        b[q] = fma(-wb, vr[q], b[q]);
      }
    }
    T* oa = d.Qc + (size_t)c0 * np;
    T* ob = d.Qc + (size_t)c1 * np;
#pragma unroll
    for (int q = 0; q < QR; ++q) {
      const int i = lane + 32 * q;
      if (i < np) {
        oa[i] = a[q];
        if (two) ob[i] = b[q];
      }
    }
  }
}

// Per reflector step k:
//   1. every warp reduces its threads' best live columns (largest squared
//      trailing norm, lowest index on ties) and pushes the result into slot
//      (rank, warp) of set k mod 2 of every CTA; barrier;
//   2. every thread reduces the C * 8 candidates: pivot j*, |R_kk| = sqrt(norm)
//      (norms are recomputed exactly each step); the truncation rule is
//      checked here, uniformly.  The owner of the previous pivot retires that
//      column now (R = beta, zeros below), every CTA having read it;
//   3. every thread derives the reflector from the raw pivot column p (read in
//      place when C == 1, else copied from the owner's shared memory into a
//      local buffer + block barrier): beta = -sign(p_k) |R_kk|,
//      tau = (beta - p_k) / beta, v = [1; p_{k+1:} / (p_k - beta)];
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
  size_t off = cq_al16(sizeof(CqShared<T>));
  CpqrNbr<T>* nbr = reinterpret_cast<CpqrNbr<T>*>(smraw + off);
  off += cq_al16((size_t)nnb * sizeof(CpqrNbr<T>));
  int* cstart = reinterpret_cast<int*>(smraw + off);
  off += cq_al16((size_t)(nnb + 1) * sizeof(int));
  T* pbuf = reinterpret_cast<T*>(smraw + off);
  off += cq_al16((size_t)L * sizeof(T));
  T* tau_s = reinterpret_cast<T*>(smraw + off);
  off += cq_al16((size_t)(np > 0 ? np : 1) * sizeof(T));
  int* tcol = reinterpret_cast<int*>(smraw + off);  // tcol[jl]: neighbour e, tcol[cpm + jl]: column in p's row
  const int cpm = d.m_max > 0 ? (d.m_max + (int)cluster.num_blocks() - 1) / (int)cluster.num_blocks() : 1;
  off += cq_al16((size_t)2 * cpm * sizeof(int));
  T* schunk = reinterpret_cast<T*>(smraw + off);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  // neighbour descriptors and their current sizes (cur_size of neighbours of
  // earlier colours already holds their ranks), loaded in parallel
  for (int e = tid; e < nnb; e += CQ_NT) {
    nbr[e] = nbrs[d.nbeg + e];
    cstart[e + 1] = cur_size[nbr[e].q];
  }
  __syncthreads();
  if (tid == 0) {
    cstart[0] = 0;
    for (int e = 0; e < nnb; ++e) cstart[e + 1] += cstart[e];
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

  // per local column: its neighbour and its column in p's block row
  for (int jl = tid; jl < nc; jl += CQ_NT) {
    const int j = j0 + jl;
    const int e = owner_nbr(j);
    tcol[jl] = e;
    tcol[cpm + jl] = nbr[e].off_pq + (j - cstart[e]);
  }
  __syncthreads();
  // ---- gather my columns of A_pn, zero the padding rows of the last vector:
  // each warp moves 8 columns at a time (lanes over rows, coalesced), with all
  // 8 loads issued before the stores
  constexpr int GU = 8;
  for (int jb = warp * GU; jb < nc; jb += CQ_NW * GU) {
    const T* src[GU];
#pragma unroll
    for (int u = 0; u < GU; ++u) src[u] = d.Rp + (size_t)tcol[cpm + min(jb + u, nc - 1)] * d.ldp;
    for (int i = lane; i < ng * VW; i += 32) {
      T v[GU];
#pragma unroll
      for (int u = 0; u < GU; ++u) v[u] = (i < np && jb + u < nc) ? src[u][i] : T(0);
#pragma unroll
      for (int u = 0; u < GU; ++u)
        if (jb + u < nc) chunk[(size_t)(jb + u) * L + i] = v[u];
    }
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
  int pj = -1, pk = 0;  // previous pivot column and its step (retired one step later)
  T pbeta = T(0);
  auto retire = [&]() {  // R_{pk,pj} = beta, zeros below, in the owner CTA
    if (pj >= j0 && pj < j0 + nc) {
      T* col = chunk + (size_t)(pj - j0) * L;
      for (int i = pk + tid; i < ng * VW; i += CQ_NT) col[i] = (i == pk) ? pbeta : T(0);
    }
    pj = -1;
  };
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
    cq_warp_argmax(bv, bj);
    if (lane < C) {  // lane q pushes this warp's candidate into CTA q
      CqShared<T>* o = C == 1 ? &sh : cluster.map_shared_rank(&sh, lane);
      o->cand_v[k & 1][rank * CQ_NW + warp] = bv;
      o->cand_j[k & 1][rank * CQ_NW + warp] = bj;
    }
    cq_sync(cluster, C);
    // 2. pivot and |R_kk| (identical in every thread of the cluster)
    T gv = T(-1);
    int gj = INT_MAX;
    for (int q = lane; q < C * CQ_NW; q += 32) {
      const T v = sh.cand_v[k & 1][q];
      const int j = sh.cand_j[k & 1][q];
      if (v > gv || (v == gv && j < gj)) {
        gv = v;
        gj = j;
      }
    }
    cq_warp_argmax(gv, gj);
    if (gj == INT_MAX) gj = 0;  // unreachable: k < kmax <= m leaves a live column
    retire();                   // every CTA finished reading the previous pivot before this barrier
    const T rkk = sqrt(gv > T(0) ? gv : T(0));
    if (k == 0) r00 = rkk;
    if (r00 == T(0) || rkk < eps * r00) {
      r = k;
      break;
    }
#pragma unroll
    for (int c = 0; c < CQ_CPT; ++c)
      if (j0 + tid + c * CQ_NT == gj) nrm[c] = T(-1);  // the pivot column leaves the live set
    // 3. the raw pivot column and the reflector
    const int owner = min(C - 1, gj / cols_per);
    const int i0 = (k / VW) * VW;
    const T* pcol;
    if (C == 1) {
      pcol = chunk + (size_t)(gj - j0) * L;
    } else {
      const size_t po = (size_t)(gj - owner * cols_per) * L;
      if (RES) {
        const T* src = cluster.map_shared_rank(schunk, owner) + po;
        for (int i = i0 + tid; i < ng * VW; i += CQ_NT) pbuf[i] = src[i];
      } else {  // the owner's chunk in global memory, written by another CTA: read through L2
        const T* src = d.gwork + (size_t)owner * L * cols_per + po;
        for (int i = i0 + tid; i < ng * VW; i += CQ_NT) pbuf[i] = __ldcg(src + i);
      }
      __syncthreads();
      pcol = pbuf;
    }
    const T alpha = pcol[k];
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
    if (tid == 0) tau_s[k] = tau;
    if (rank == owner)  // v_k for the formation of Q_pc
      for (int i = k + tid; i < np; i += CQ_NT) d.V[i + (size_t)k * np] = (i == k) ? T(1) : pcol[i] * scal;
    pj = gj;
    pk = k;
    pbeta = beta;
    // 4. apply H_k = I - tau v v^T to my live columns, recompute their trailing norms:
    //    w = tau (x_k + scal p_{k+1:}^T x_{k+1:}),  x_k -= w,  x_{k+1:} -= (w scal) p_{k+1:}
    const int gs = k / VW;
    const int rb = gs * VW;
    const V* __restrict__ pv = reinterpret_cast<const V*>(pcol);
#pragma unroll
    for (int c = 0; c < CQ_CPT; ++c) {
      if (nrm[c] < T(0)) continue;
      T* colp = chunk + (size_t)(tid + c * CQ_NT) * L;
      V* __restrict__ cv = reinterpret_cast<V*>(colp);
      T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
      {  // first vector: only rows > k
        const V x = cv[gs], p = pv[gs];
        if (rb > k) a0 = x.x * p.x;
        if (rb + 1 > k) a1 = x.y * p.y;
        if constexpr (VW == 4) {
          if (rb + 2 > k) a2 = x.z * p.z;
          if (rb + 3 > k) a3 = x.w * p.w;
        }
      }
#pragma unroll 2
      for (int g = gs + 1; g < ng; ++g) {
        const V x = cv[g], p = pv[g];
        a0 = fma(x.x, p.x, a0);
        a1 = fma(x.y, p.y, a1);
        if constexpr (VW == 4) {
          a2 = fma(x.z, p.z, a2);
          a3 = fma(x.w, p.w, a3);
        }
      }
      const T w = tau * fma(scal, (a0 + a1) + (a2 + a3), colp[k]);
      const T ws = w * scal;
      T q0 = 0, q1 = 0, q2 = 0, q3 = 0;
      {  // first vector: row k takes -w, rows > k take -ws p and enter the norm
        V x = cv[gs];
        const V p = pv[gs];
        if (rb == k) x.x -= w;
        else if (rb > k) { x.x = fma(-ws, p.x, x.x); q0 = x.x * x.x; }
        if (rb + 1 == k) x.y -= w;
        else if (rb + 1 > k) { x.y = fma(-ws, p.y, x.y); q1 = x.y * x.y; }
        if constexpr (VW == 4) {
          if (rb + 2 == k) x.z -= w;
          else if (rb + 2 > k) { x.z = fma(-ws, p.z, x.z); q2 = x.z * x.z; }
          if (rb + 3 == k) x.w -= w;
          else if (rb + 3 > k) { x.w = fma(-ws, p.w, x.w); q3 = x.w * x.w; }
        }
        cv[gs] = x;
      }
#pragma unroll 2
      for (int g = gs + 1; g < ng; ++g) {
        V x = cv[g];
        const V p = pv[g];
        x.x = fma(-ws, p.x, x.x);
        x.y = fma(-ws, p.y, x.y);
        q0 = fma(x.x, x.x, q0);
        q1 = fma(x.y, x.y, q1);
        if constexpr (VW == 4) {
          x.z = fma(-ws, p.z, x.z);
          x.w = fma(-ws, p.w, x.w);
          q2 = fma(x.z, x.z, q2);
          q3 = fma(x.w, x.w, q3);
        }
        cv[g] = x;
      }
      nrm[c] = (q0 + q1) + (q2 + q3);
    }
  }
  __syncthreads();  // every thread is done with the last pivot column
  retire();         // the last pivot when the loop ran to kmax
  __syncthreads();
  // Rows 0..r-1 of every column now hold W_cn in the original column order
  // (the pivot found at step r, if any, was not touched).
  // ---- write back W_cn into p's row (one warp per column, coalesced) ...
  for (int jl = warp; jl < nc; jl += CQ_NW) {
    T* dst = d.Rp + (size_t)tcol[cpm + jl] * d.ldp;
    const T* src = chunk + (size_t)jl * L;
    for (int i = lane; i < r; i += 32) dst[i] = src[i];
  }
  // ... and its transpose into the neighbours' rows (one thread per column)
  for (int jl = tid; jl < nc; jl += CQ_NT) {
    const int e = tcol[jl];
    const CpqrNbr<T> nb = nbr[e];
    const int cc = j0 + jl - cstart[e];
    const T* src = chunk + (size_t)jl * L;
    for (int i = 0; i < r; ++i) nb.Rq[cc + (size_t)(nb.off_qp + i) * nb.ldq] = src[i];
  }
  // A_cc = I: column j by warp j of the cluster, lanes over rows
  for (int j = rank * CQ_NW + warp; j < r; j += C * CQ_NW) {
    T* dst = d.Rp + (size_t)j * d.ldp;
    for (int i = lane; i < r; i += 32) dst[i] = (i == j) ? T(1) : T(0);
  }
  if (C > 1) cluster.sync();  // every V column is visible cluster-wide
  else __syncthreads();
  // ---- Q_pc e_c = H_0 ... H_c e_c (H_k e_c = e_c for k > c), one warp per
  // column, the column held in registers (lane l owns rows l, l+32, ...).  The
  // reflectors are read from a shared-memory copy of V when it fits in the
  // chunk's space (free again after the write-back).
  const T* Vsrc = d.V;
  if (RES && (size_t)np * r <= (size_t)L * cols_per) {
    // V was written by other CTAs: read through L2; 8 columns per warp in flight
    T* Vs = schunk;
    for (int kb = warp * 8; kb < r; kb += CQ_NW * 8)
      for (int i = lane; i < np; i += 32) {
        T v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = (kb + u < r && i >= kb + u) ? __ldcg(d.V + i + (size_t)(kb + u) * np) : T(0);
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (kb + u < r) Vs[i + (size_t)(kb + u) * np] = v[u];
      }
    __syncthreads();
    Vsrc = Vs;
  }
  if (np > 32 * 16) {  // tall interfaces: the column lives in global memory
    for (int c = rank * CQ_NW + warp; c < r; c += C * CQ_NW) {
      T* col = d.Qc + (size_t)c * np;
      for (int i = lane; i < np; i += 32) col[i] = (i == c) ? T(1) : T(0);
      __syncwarp();
      for (int k = c; k >= 0; --k) {
        const T tk = tau_s[k];
        if (tk == T(0)) continue;
        const T* v = Vsrc + (size_t)k * np;
        T w = 0;
        for (int i = k + lane; i < np; i += 32) w += __ldcg(v + i) * col[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        w *= tk;
        for (int i = k + lane; i < np; i += 32) col[i] -= w * __ldcg(v + i);
        __syncwarp();
      }
    }
  } else if (np > 32 * 8) {
    cq_form_q<T, 16>(d, Vsrc, tau_s, r, np, rank, C);
  } else if (np > 32 * 4) {
    cq_form_q<T, 8>(d, Vsrc, tau_s, r, np, rank, C);
  } else if (np > 32 * 2) {
    cq_form_q<T, 4>(d, Vsrc, tau_s, r, np, rank, C);
  } else if (np > 32) {
    cq_form_q<T, 2>(d, Vsrc, tau_s, r, np, rank, C);
  } else {
    cq_form_q<T, 1>(d, Vsrc, tau_s, r, np, rank, C);
  }
  if (rank == 0 && tid == 0) cur_size[d.p] = r;
  if (C > 1) cluster.sync();  // no CTA leaves while others may still read its shared memory
}

}  // namespace spand

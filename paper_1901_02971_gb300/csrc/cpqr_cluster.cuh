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
// Columns are never swapped and a pivot column is never written again: its
// entries below the diagonal keep the raw values p from which the Householder
// vector is derived (v = [1; p / (p_k - beta)]), so the reflectors need no
// storage of their own; the write-back emits R_kk = beta and zeros below for
// retired columns.  Per reflector step the CTAs of a cluster exchange their
// pivot candidates, each with its column, through distributed shared memory:
// one block barrier per step plus one cluster barrier when C > 1, no
// spin-waits.
#pragma once

#include <cooperative_groups.h>

#include "dense_tiles.cuh"

namespace spand {

namespace cg = cooperative_groups;

constexpr int CQ_MAXNT = 512;              // threads per CTA: 256 or 512 (chosen per launch)
constexpr int CQ_MAXW = CQ_MAXNT / 32;
constexpr int CQ_MAXC = 16;         // largest cluster
constexpr int CQ_CPT = 4;           // columns per thread group at most (the host sizes clusters for it)

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
  T* tau;             // np: tau_k of the reflectors, for k_form_q
  T* Qc;              // np x np capacity; first r columns = Q_pc after k_form_q
  int32_t* rank_out;  // where the rank goes; nullptr: the cur_size array the sizes are read from
  int32_t p, np, ldp, nbeg, nend, m_max;
  int32_t nowb;       // 1: leave the blocks untouched (no W_cn write-back, simultaneous order)
};

// Destination of the rank of task d: a separate array when every interface of
// a level is sparsified from the same matrix (the neighbours' sizes must not
// change while the launch reads them), else the size array itself.
template <typename T>
__device__ __forceinline__ int32_t* cq_rank_dst(const CpqrTask<T>& d, int32_t* cur_size) {
  return d.rank_out ? d.rank_out : cur_size;
}

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
  // pivot candidates, double-buffered by step parity (a fast warp or CTA
  // writes step k+1 while a slow one may still read step k): with C == 1 one
  // slot per warp; with C > 1 the warps' slots feed a CTA-level reduction and
  // slot q of cta_v/cta_j holds the best of CTA q (pushed by it)
  T cand_v[2][CQ_MAXW];
  int cand_j[2][CQ_MAXW];
  T cta_v[2][CQ_MAXC];
  int cta_j[2][CQ_MAXC];
};

__host__ __device__ inline size_t cq_al16(size_t b) { return (b + 15) & ~size_t(15); }

// Fixed shared memory before the chunk, each part 16-byte aligned: CqShared,
// the neighbour descriptors (nnb), their column starts (nnb + 1 ints), the
// candidate columns pushed by the cluster's CTAs (2 x C x L elements, none
// when C == 1), per reflector its pivot column, beta, tau and scale (np
// each), and per local column its neighbour, its column in p's block row and
// the step at which it became the pivot (3 cols_per ints).
template <typename T>
__host__ __device__ inline size_t cq_fixed_smem(int nnb, int np, int cols_per, int C) {
  const size_t npp = (size_t)(np > 0 ? np : 1), cp = (size_t)(cols_per > 0 ? cols_per : 1);
  const size_t cand = C > 1 ? (size_t)2 * C * cq_ld<T>(np) : 0;
  return cq_al16(sizeof(CqShared<T>)) + cq_al16((size_t)nnb * sizeof(CpqrNbr<T>)) +
         cq_al16((size_t)(nnb + 1) * sizeof(int)) + cq_al16(cand * sizeof(T)) + 3 * cq_al16(npp * sizeof(T)) +
         cq_al16(npp * sizeof(int)) + cq_al16(3 * cp * sizeof(int));
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
// this warp (warp w of block `rank` out of C blocks takes the column pairs
// (c, c + C NW) with c = rank NW + w mod 2 C NW), the column held in
// registers: lane l owns rows l + 32 q, q < QR (np <= 32 QR).  Reflector k is
// read from column k of V (rows >= k; v_k[k] = 1).
template <typename T, int QR>
__device__ __forceinline__ void cq_form_q(const CpqrTask<T>& d, const T* V, const T* tau_s, int r, int np, int rank,
                                          int C) {
  // two columns per warp, their reflector chains interleaved (independent
  // shuffle reductions); c1 > c0, so H_k for c0 < k <= c1 touches c1 only
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwc = (int)(blockDim.x >> 5), nwarps = C * nwc, w0 = rank * nwc + warp;
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
      T vr[QR];
      const T* v = V + (size_t)k * np;
#pragma unroll
      for (int q = 0; q < QR; ++q) {
        const int i = lane + 32 * q;
        vr[q] = (i >= k && i < np) ? v[i] : T(0);
      }
      T wa = 0, wb = 0;
#pragma unroll
      for (int q = 0; q < QR; ++q) {
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

template <typename T>
__device__ __forceinline__ void cq_form_q_any(const CpqrTask<T>& d, const T* V, const T* tau_s, int r, int np,
                                              int rank, int C) {
  if (np > 32 * 8) cq_form_q<T, 16>(d, V, tau_s, r, np, rank, C);
  else if (np > 32 * 4) cq_form_q<T, 8>(d, V, tau_s, r, np, rank, C);
  else if (np > 32 * 2) cq_form_q<T, 4>(d, V, tau_s, r, np, rank, C);
  else if (np > 32) cq_form_q<T, 2>(d, V, tau_s, r, np, rank, C);
  else cq_form_q<T, 1>(d, V, tau_s, r, np, rank, C);
}

// Epilogue shared by the sparsification kernels, entered after a block barrier
// with the CTA's final columns in `chunk` (column-major, stride L): the write-back
// of W_cn into p's and the neighbours' block rows, A_cc = I, the reflectors
// (V, tau) from which k_form_q forms Q_pc, and the rank in cur_size[p] (or
// the task's rank_out); with nowb the blocks are left as they are.
template <typename T, int NT>
__device__ __forceinline__ void cq_finish(const CpqrTask<T>& d, cg::cluster_group& cluster, int C, int rank,
                                          const T* chunk, int L, int np, int r, int nc, int j0,
                                          int cpm, const int* tcol, const int* rstep,
                                          const T* beta_s, const T* scal_s, const T* tau_s, const int* piv_s,
                                          const CpqrNbr<T>* nbr, const int* cstart, int32_t* cur_size) {
  constexpr int NW = NT / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // Rows 0..r-1 of every column hold W_cn in the original column order, except
  // that a column retired at step s < r holds R_ss = beta_s at row s and zeros
  // below it (its stored entries below s are the raw reflector source).
  auto wval = [&](int jl, int i) -> T {
    const int s = rstep[jl];
    if (s < 0 || i < s) return chunk[(size_t)jl * L + i];
    return i == s ? beta_s[s] : T(0);
  };
  // ---- write back W_cn into p's row (one warp per column, coalesced) ...
  const int nwb = d.nowb ? 0 : nc;
  for (int jl = warp; jl < nwb; jl += NW) {
    T* dst = d.Rp + (size_t)tcol[cpm + jl] * d.ldp;
    for (int i = lane; i < r; i += 32) dst[i] = wval(jl, i);
  }
  // ... and its transpose into the neighbours' rows (one thread per column)
  for (int jl = tid; jl < nwb; jl += NT) {
    const int e = tcol[jl];
    const CpqrNbr<T> nb = nbr[e];
    const int cc = j0 + jl - cstart[e];
    for (int i = 0; i < r; ++i) nb.Rq[cc + (size_t)(nb.off_qp + i) * nb.ldq] = wval(jl, i);
  }
  // A_cc = I: column j by warp j of the cluster, lanes over rows (not with
  // nowb: the block row is then left as it is -- its scaled diagonal block
  // is I already, or it is the sketch of the randomized compression, whose
  // leading columns the next, wider round reuses)
  for (int j = rank * NW + warp; j < (d.nowb ? 0 : r); j += C * NW) {
    T* dst = d.Rp + (size_t)j * d.ldp;
    for (int i = lane; i < r; i += 32) dst[i] = (i == j) ? T(1) : T(0);
  }
  // ---- the reflectors, for k_form_q: v_k (rows >= k, v_k[k] = 1) into
  // column k of V by the CTA that holds pivot column k, tau by rank 0
  for (int k = warp; k < r; k += NW) {
    const int jl = piv_s[k] - j0;
    if (jl < 0 || jl >= nc) continue;
    const T* pc = chunk + (size_t)jl * L;
    const T sc = scal_s[k];
    for (int i = k + lane; i < np; i += 32) d.V[i + (size_t)k * np] = i == k ? T(1) : pc[i] * sc;
  }
  if (rank == 0)
    for (int k = tid; k < r; k += NT) d.tau[k] = tau_s[k];
  if (rank == 0 && tid == 0) cq_rank_dst(d, cur_size)[d.p] = r;
  if (C > 1) cluster.sync();  // no CTA leaves while another may still address its shared memory
}

// Per reflector step k:
//   1. every warp reduces its threads' best live columns (largest squared
//      trailing norm, lowest index on ties) into its slot of set k mod 2;
//      block barrier; every warp reduces the slots to the CTA's candidate;
//      with C > 1 each CTA pushes its candidate and that column's rows >= k
//      into every CTA of the cluster; cluster barrier;
//   2. every thread reduces the C candidates: pivot j*, |R_kk| = sqrt(norm)
//      (norms are recomputed exactly each step); the truncation rule is
//      checked here, uniformly;
//   3. every thread derives the reflector from the raw pivot column p (read in
//      place when C == 1, else from the copy its owner pushed):
//      beta = -sign(p_k) |R_kk|,
//      tau = (beta - p_k) / beta, v = [1; p_{k+1:} / (p_k - beta)];
//   4. every thread applies H_k to its live columns and recomputes their
//      trailing norms.
//
// Column ownership: with LG lanes per column, thread t belongs to group
// t / LG, which owns the local columns t / LG + c * (NT / LG), c < CQ_CPT;
// lane t % LG of the group takes the vectors gs + lane, gs + lane + LG, ...
// of a column (gs: the vector holding row k), and the group's partial dot
// products and norms are summed over its lanes with xor shuffles (every lane
// ends with the same bits).  LG > 1 spends otherwise idle threads of a CTA
// with fewer columns than threads on shortening each step's per-column
// sweep, which is the step's latency.
template <int LG, typename T>
__device__ __forceinline__ T cq_group_sum(T v) {
  if constexpr (LG > 1) {
    const unsigned lane = threadIdx.x & 31;
    const unsigned mask = ((1u << LG) - 1u) << (lane & ~(unsigned)(LG - 1));
#pragma unroll
    for (int o = 1; o < LG; o <<= 1) v += __shfl_xor_sync(mask, v, o);
  }
  return v;
}

template <typename T, bool RES, int NT, int LG = 1>
__global__ void __launch_bounds__(NT) k_cpqr_cluster(const CpqrTask<T>* __restrict__ tasks,
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
  const int npp = np > 0 ? np : 1;
  const int cpm = d.m_max > 0 ? (d.m_max + C - 1) / C : 1;  // host bound on the columns per CTA
  extern __shared__ __align__(16) unsigned char smraw[];
  CqShared<T>& sh = *reinterpret_cast<CqShared<T>*>(smraw);
  size_t off = cq_al16(sizeof(CqShared<T>));
  CpqrNbr<T>* nbr = reinterpret_cast<CpqrNbr<T>*>(smraw + off);
  off += cq_al16((size_t)nnb * sizeof(CpqrNbr<T>));
  int* cstart = reinterpret_cast<int*>(smraw + off);
  off += cq_al16((size_t)(nnb + 1) * sizeof(int));
  T* cbuf = reinterpret_cast<T*>(smraw + off);  // [parity][source CTA][L]: candidate columns
  off += cq_al16((C > 1 ? (size_t)2 * C * L : 0) * sizeof(T));
  T* tau_s = reinterpret_cast<T*>(smraw + off);
  off += cq_al16((size_t)npp * sizeof(T));
  T* beta_s = reinterpret_cast<T*>(smraw + off);
  off += cq_al16((size_t)npp * sizeof(T));
  T* scal_s = reinterpret_cast<T*>(smraw + off);
  off += cq_al16((size_t)npp * sizeof(T));
  int* piv_s = reinterpret_cast<int*>(smraw + off);
  off += cq_al16((size_t)npp * sizeof(int));
  int* tcol = reinterpret_cast<int*>(smraw + off);  // [0, cpm): neighbour; [cpm, 2cpm): column in p's row;
  off += cq_al16((size_t)3 * cpm * sizeof(int));    // [2cpm, 3cpm): step at which the column was the pivot (-1)
  T* schunk = reinterpret_cast<T*>(smraw + off);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = NT / 32;
  constexpr int NG = NT / LG;             // column groups
  const int grp = tid / LG, lg = tid % LG;

  // neighbour descriptors and their current sizes (cur_size of neighbours of
  // earlier colours already holds their ranks), loaded in parallel
  for (int e = tid; e < nnb; e += NT) {
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
  if (m == 0) {  // every neighbour reduced to nothing: p is kept as it is (Q_pc = I, all tau = 0)
    if (rank == 0) {
      for (int k = tid; k < np; k += NT) d.tau[k] = T(0);
      if (tid == 0) cq_rank_dst(d, cur_size)[d.p] = np;
    }
    return;  // uniform across the cluster (m is the same for every CTA)
  }
  const int cols_per = (m + C - 1) / C;
  const int j0 = min(m, rank * cols_per);
  const int nc = min(m, j0 + cols_per) - j0;
  T* __restrict__ chunk = RES ? schunk : d.gwork + (size_t)rank * L * cols_per;
  int* rstep = tcol + 2 * cpm;

  // per local column: its neighbour (binary search over the column starts) and
  // its column in p's block row
  for (int jl = tid; jl < nc; jl += NT) {
    const int j = j0 + jl;
    int lo = 0, hi = nnb - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (cstart[mid] <= j) lo = mid; else hi = mid - 1;
    }
    tcol[jl] = lo;
    tcol[cpm + jl] = nbr[lo].off_pq + (j - cstart[lo]);
    rstep[jl] = -1;
  }
  __syncthreads();
  // ---- gather my columns of A_pn, zero the padding rows of the last vector:
  // each warp moves 8 columns at a time (lanes over rows, coalesced), with all
  // 8 loads issued before the stores
  constexpr int GU = 8;
  for (int jb = warp * GU; jb < nc; jb += NW * GU) {
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
  // squared norms of my columns (-1: retired or absent)
  T nrm[CQ_CPT];
#pragma unroll
  for (int c = 0; c < CQ_CPT; ++c) {
    const int jl = grp + c * NG;
    nrm[c] = T(-1);
    if (jl < nc) {  // uniform over the group
      const V* cv = reinterpret_cast<const V*>(chunk + (size_t)jl * L);
      T s = 0;
      for (int g = lg; g < ng; g += LG) {
        const V x = cv[g];
        if constexpr (VW == 4) s += x.x * x.x + x.y * x.y + x.z * x.z + x.w * x.w;
        else s += x.x * x.x + x.y * x.y;
      }
      nrm[c] = cq_group_sum<LG>(s);
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
        bj = j0 + grp + c * NG;
      }
    cq_warp_argmax(bv, bj);
    if (lane == 0) {
      sh.cand_v[k & 1][warp] = bv;
      sh.cand_j[k & 1][warp] = bj;
    }
    __syncthreads();
    // 2. pivot and |R_kk| (identical in every thread of the cluster)
    T gv = lane < NW ? sh.cand_v[k & 1][lane] : T(-1);
    int gj = lane < NW ? sh.cand_j[k & 1][lane] : INT_MAX;
    cq_warp_argmax(gv, gj);
    const int i0 = (k / VW) * VW;
    if (C > 1) {
      // one candidate per CTA crosses the cluster, with its column (rows
      // >= i0), so that the winner's column is local after the barrier
      if (gj != INT_MAX) {
        const T* src = chunk + (size_t)(gj - j0) * L;
        for (int i = i0 + tid; i < ng * VW; i += NT) {
          const T v = src[i];
          for (int q = 0; q < C; ++q) cluster.map_shared_rank(cbuf, q)[((size_t)(k & 1) * C + rank) * L + i] = v;
        }
      }
      if (warp == 0 && lane < C) {
        CqShared<T>* o = cluster.map_shared_rank(&sh, lane);
        o->cta_v[k & 1][rank] = gv;
        o->cta_j[k & 1][rank] = gj;
      }
      cluster.sync();
      gv = lane < C ? sh.cta_v[k & 1][lane] : T(-1);
      gj = lane < C ? sh.cta_j[k & 1][lane] : INT_MAX;
      cq_warp_argmax(gv, gj);
    }
    if (gj == INT_MAX) gj = 0;  // unreachable: k < kmax <= m leaves a live column
    const T rkk = sqrt(gv > T(0) ? gv : T(0));
    if (k == 0) r00 = rkk;
    if (r00 == T(0) || rkk < eps * r00) {
      r = k;
      break;
    }
#pragma unroll
    for (int c = 0; c < CQ_CPT; ++c)
      if (j0 + grp + c * NG == gj) nrm[c] = T(-1);  // the pivot column leaves the live set
    // 3. the raw pivot column (never written again) and the reflector
    const T* pcol = C == 1 ? chunk + (size_t)(gj - j0) * L
                           : cbuf + ((size_t)(k & 1) * C + min(C - 1, gj / cols_per)) * L;
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
    if (tid == 0) {
      tau_s[k] = tau;
      beta_s[k] = beta;
      scal_s[k] = scal;
      piv_s[k] = gj;
    }
    if (gj >= j0 && gj < j0 + nc && tid == 0) rstep[gj - j0] = k;
    // 4. apply H_k = I - tau v v^T to my live columns, recompute their trailing norms:
    //    w = tau (x_k + scal p_{k+1:}^T x_{k+1:}),  x_k -= w,  x_{k+1:} -= (w scal) p_{k+1:}
    const int gs = k / VW;
    const int rb = gs * VW;
    const V* __restrict__ pv = reinterpret_cast<const V*>(pcol);
#pragma unroll
    for (int c = 0; c < CQ_CPT; ++c) {
      if (nrm[c] < T(0)) continue;  // uniform over the group
      T* colp = chunk + (size_t)(grp + c * NG) * L;
      V* __restrict__ cv = reinterpret_cast<V*>(colp);
      const T xk = colp[k];
      if constexpr (LG > 1) {
        // the group's lanes take interleaved vectors; lane 0 holds vector gs
        T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
        for (int g = gs + lg; g < ng; g += LG) {
          const V x = cv[g], p = pv[g];
          if (g == gs) {
            if (rb > k) a0 = fma(x.x, p.x, a0);
            if (rb + 1 > k) a1 = fma(x.y, p.y, a1);
            if constexpr (VW == 4) {
              if (rb + 2 > k) a2 = fma(x.z, p.z, a2);
              if (rb + 3 > k) a3 = fma(x.w, p.w, a3);
            }
          } else {
            a0 = fma(x.x, p.x, a0);
            a1 = fma(x.y, p.y, a1);
            if constexpr (VW == 4) {
              a2 = fma(x.z, p.z, a2);
              a3 = fma(x.w, p.w, a3);
            }
          }
        }
        const T dot = cq_group_sum<LG>((a0 + a1) + (a2 + a3));
        const T w = tau * fma(scal, dot, xk);
        const T ws = w * scal;
        T q0 = 0, q1 = 0, q2 = 0, q3 = 0;
        for (int g = gs + lg; g < ng; g += LG) {
          V x = cv[g];
          const V p = pv[g];
          if (g == gs) {  // row k takes -w, rows > k take -ws p and enter the norm
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
          } else {
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
          }
          cv[g] = x;
        }
        nrm[c] = cq_group_sum<LG>((q0 + q1) + (q2 + q3));
        continue;
      }
      T a0 = 0, a1 = 0, a2 = 0, a3 = 0, b0 = 0, b1 = 0, b2 = 0, b3 = 0;
      {  // first vector: only rows > k
        const V x = cv[gs], p = pv[gs];
        if (rb > k) a0 = x.x * p.x;
        if (rb + 1 > k) a1 = x.y * p.y;
        if constexpr (VW == 4) {
          if (rb + 2 > k) a2 = x.z * p.z;
          if (rb + 3 > k) a3 = x.w * p.w;
        }
      }
      int g = gs + 1;
      for (; g + 1 < ng; g += 2) {  // two vectors per trip, independent accumulators
        const V x0 = cv[g], p0 = pv[g], x1 = cv[g + 1], p1 = pv[g + 1];
        a0 = fma(x0.x, p0.x, a0);
        a1 = fma(x0.y, p0.y, a1);
        b0 = fma(x1.x, p1.x, b0);
        b1 = fma(x1.y, p1.y, b1);
        if constexpr (VW == 4) {
          a2 = fma(x0.z, p0.z, a2);
          a3 = fma(x0.w, p0.w, a3);
          b2 = fma(x1.z, p1.z, b2);
          b3 = fma(x1.w, p1.w, b3);
        }
      }
      if (g < ng) {
        const V x0 = cv[g], p0 = pv[g];
        a0 = fma(x0.x, p0.x, a0);
        a1 = fma(x0.y, p0.y, a1);
        if constexpr (VW == 4) {
          a2 = fma(x0.z, p0.z, a2);
          a3 = fma(x0.w, p0.w, a3);
        }
      }
      const T dot = ((a0 + b0) + (a1 + b1)) + ((a2 + b2) + (a3 + b3));
      const T w = tau * fma(scal, dot, xk);
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
      for (g = gs + 1; g < ng; ++g) {
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
  __syncthreads();
  cq_finish<T, NT>(d, cluster, C, rank, chunk, L, np, r, nc, j0, cpm, tcol, rstep, beta_s, scal_s, tau_s, piv_s,
                   nbr, cstart, cur_size);
}


// Q_pc = H_0 ... H_{r-1} [I_r; 0] (Sec. 2.6.1) of interfaces whose QR kernel
// has finished, from the reflectors it left in V and tau and the rank in
// cur_size[p] (or in the task's rank_out).  Launched per colour on a side stream, so that it overlaps the
// next colour's QR; it is off the sparsification's critical path.  Block b of
// an interface (nb blocks each) takes the column pairs (c, c + nb NW) with
// c = b NW + warp (mod 2 nb NW), so every block meets chains of every length;
// V is copied into shared memory when it fits (smem_elems elements).
template <typename T, int NT>
__global__ void __launch_bounds__(NT) k_form_q(const CpqrTask<T>* __restrict__ tasks,
                                                 const int32_t* __restrict__ list,
                                                 const int32_t* __restrict__ cur_size, int nb, int smem_elems) {
  constexpr int NW = NT / 32;
  const CpqrTask<T> d = tasks[list[blockIdx.x / nb]];
  const int b = blockIdx.x % nb;
  const int np = d.np, r = d.rank_out ? d.rank_out[d.p] : cur_size[d.p];
  if (r <= 0 || b * NW >= r) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* tau_s = reinterpret_cast<T*>(smraw);
  T* vs = tau_s + cq_al16((size_t)r * sizeof(T)) / sizeof(T);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int k = tid; k < r; k += NT) tau_s[k] = d.tau[k];
  const T* Vsrc = d.V;
  const size_t nv = (size_t)np * r;
  if (np <= 32 * 16 && (size_t)(vs - tau_s) + nv <= (size_t)smem_elems) {
    for (size_t e = tid; e < nv; e += NT) vs[e] = __ldcg(d.V + e);  // rows < k of column k are never read
    Vsrc = vs;
  }
  __syncthreads();
  if (np <= 32 * 16) {
    cq_form_q_any<T>(d, Vsrc, tau_s, r, np, b, nb);
    return;
  }
  // tall interfaces: one warp per column, V and the column in global memory
  for (int c = b * NW + warp; c < r; c += nb * NW) {
    T* col = d.Qc + (size_t)c * np;
    for (int i = lane; i < np; i += 32) col[i] = (i == c) ? T(1) : T(0);
    __syncwarp();
    for (int k = c; k >= 0; --k) {
      const T tk = tau_s[k];
      if (tk == T(0)) continue;
      const T* v = d.V + (size_t)k * np;
      T w = 0;
      for (int i = k + lane; i < np; i += 32) w += __ldcg(v + i) * col[i];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
      w *= tk;
      for (int i = k + lane; i < np; i += 32) col[i] -= w * __ldcg(v + i);
      __syncwarp();
    }
  }
}

}  // namespace spand

// Register-resident orthogonal sparsification of scaled interfaces (Sec. 2.6.1,
// truncation rule of Sec. 4): the same task, pivot rule, result and write-back
// as k_cpqr_cluster, for interfaces whose coupling A_pn fits in the registers
// of one cluster.
//
// GB300 mapping: G consecutive lanes own one column of A_pn; lane g of the
// group keeps rows g, g + G, ..., g + (R - 1) G of it in registers (slot q is
// row q G + g).  A reflector step then reads no memory but the pivot column:
// the dot product, the update and the trailing norm are register FMAs, reduced
// over the group with xor shuffles (every lane of a group ends with the same
// bits).  Slots are processed in chunks of 8; a chunk whose rows all lie above
// the current step k, or at or beyond np, is skipped, uniformly over the
// cluster, so the work per step follows the trailing rows.
//
// Pivot column: before the step's block barrier the group holding the warp's
// candidate derives the reflector it would define (alpha, beta and
// gam = 1 / (beta (beta - alpha)), so that H_k = I - gam u u^T) and writes u
// into the warp's pivot slot: its live chunks, lane-major (lane g's slots
// contiguous, segment stride R + one 16-byte vector, so that the lanes of a
// group read distinct bank groups and the groups of a warp share them by
// broadcast), with zeros above row k and alpha - beta at row k; dot product
// and update then run unmasked over the live chunks.  With C > 1 every CTA
// stores its record and winning slot into each CTA of the cluster with
// st.async, which counts the bytes on the receiver's mbarrier for that step
// parity; one thread per CTA waits (bounded) for the C records and slots, and
// a block barrier hands them and the outcome to the CTA: one block barrier
// plus one mbarrier wait per step, no cluster barrier.
//
// A retired pivot column keeps the raw values from which its reflector is
// derived; at the end every group stores its column into the shared chunk
// (column-major, stride cq_ld(np)) and the chunked kernel's epilogue writes
// W_cn, A_cc = I and the reflectors (Q_pc is formed by k_form_q).
#pragma once

#include <type_traits>

#include "cpqr_cluster.cuh"

namespace spand {

// Sum over the G lanes of an aligned lane group (identical bits in every lane:
// each butterfly level adds the same two partial sums, in commuted order).
template <int G, typename T>
__device__ __forceinline__ T cqr_group_sum(T v, unsigned mask) {
#pragma unroll
  for (int o = 1; o < G; o <<= 1) v += __shfl_xor_sync(mask, v, o);
  return v;
}

template <typename T, int G, int R>
struct CqrShape {
  static constexpr int VW = 16 / (int)sizeof(T);  // elements per 16-byte vector
  static constexpr int RS = R + VW;               // lane segment stride in a pivot slot
  static constexpr int SL = G * RS;               // pivot slot length (elements)
  static constexpr int NCH = R / 8;               // chunks of 8 slots
};

// A pivot candidate: squared trailing norm v, column j, and its reflector
// (alpha = the column's entry at row k, beta = -sign(alpha) sqrt(v),
// gam = 1 / (beta (beta - alpha)), so that H_k = I - gam u u^T with
// u = [0; alpha - beta; rows > k]).
template <typename T>
struct __align__(16) CqrRec {
  T v, a, b, gam;
  int j, pad0, pad1, pad2;
};

template <typename T>
struct CqrShared {
  CqrRec<T> w[2][CQ_MAXW];  // per warp, by step parity
  CqrRec<T> c[2][CQ_MAXC];  // per CTA of the cluster (sent by it), by step parity
  unsigned long long bar[2];  // per step parity: arrival of the C records and pivot slots
};

// Cluster exchange without a cluster barrier: every CTA stores its candidate
// record and pivot slot into each CTA of the cluster with st.async, which
// counts the bytes on the receiving CTA's mbarrier for that step parity; a CTA
// proceeds once its own mbarrier phase completes.
__device__ __forceinline__ unsigned cqr_smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned cqr_mapa(unsigned addr, unsigned rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
__device__ __forceinline__ void cqr_st_async(unsigned raddr, uint4 v, unsigned rbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, [%5];"
               :: "r"(raddr), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w), "r"(rbar) : "memory");
}
__device__ __forceinline__ void cqr_bar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(cqr_smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void cqr_bar_expect(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(cqr_smem_addr(bar)), "r"(bytes)
               : "memory");
}
constexpr long long kCqrWaitCycles = 1ll << 31;  // about a second: a wait that long is an error
// Waits for the completion of the phase with the given parity; false after
// kCqrWaitCycles without it (the caller then leaves the step loop, uniformly
// over its CTA, and reports the rank as -2).
__device__ __forceinline__ bool cqr_bar_wait(unsigned long long* bar, unsigned parity) {
  const unsigned a = cqr_smem_addr(bar);
  const long long t0 = clock64();
  for (;;) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok) : "r"(a), "r"(parity) : "memory");
    if (ok) return true;
    if (clock64() - t0 > kCqrWaitCycles) return false;
  }
}

// Chunk dispatch with compile-time chunk indices (register arrays stay in
// registers): cqr_chunks calls f(c) for c = c0, ..., c1 - 1 by a jump into a
// fall-through chain, cqr_chunk calls f(c0) alone.  Both branch on the
// (cluster-uniform) bounds instead of predicating every chunk.
#define CQR_RUN(c)                             \
  case c:                                      \
    if constexpr (c < NCH) {                   \
      if (c >= c1) break;                      \
      f(std::integral_constant<int, c>{});     \
    }                                          \
    [[fallthrough]];
template <int NCH, typename F>
__device__ __forceinline__ void cqr_chunks(int c0, int c1, F&& f) {
  static_assert(NCH <= 8, "");
  switch (c0) {
    CQR_RUN(0) CQR_RUN(1) CQR_RUN(2) CQR_RUN(3) CQR_RUN(4) CQR_RUN(5) CQR_RUN(6) CQR_RUN(7)
    default: break;
  }
}
#undef CQR_RUN
#define CQR_ONE(c)                             \
  case c:                                      \
    if constexpr (c < NCH) f(std::integral_constant<int, c>{}); \
    break;
template <int NCH, typename F>
__device__ __forceinline__ void cqr_chunk(int c0, F&& f) {
  static_assert(NCH <= 8, "");
  switch (c0) {
    CQR_ONE(0) CQR_ONE(1) CQR_ONE(2) CQR_ONE(3) CQR_ONE(4) CQR_ONE(5) CQR_ONE(6) CQR_ONE(7)
    default: break;
  }
}
#undef CQR_ONE

// Dynamic shared memory of k_cpqr_reg: the fixed part of the chunked kernel
// (without its candidate columns), the candidate records, then one region that
// holds first the staging chunk (cols_per columns of stride cq_ld(np)) and
// during the steps the pivot slots (2 x NW warp slots, and 2 x C pushed slots
// when C > 1).
template <typename T, int NT, int G, int R>
__host__ __device__ inline size_t cqr_smem(int nnb, int np, int cols_per, int C) {
  typedef CqrShape<T, G, R> S;
  const size_t stage = (size_t)cq_ld<T>(np) * (size_t)(cols_per > 0 ? cols_per : 1);
  const size_t slots = (size_t)S::SL * (2 * (NT / 32) + (C > 1 ? 2 * C : 0));
  return cq_fixed_smem<T>(nnb, np, cols_per, 1) + cq_al16(sizeof(CqrShared<T>)) +
         (stage > slots ? stage : slots) * sizeof(T);
}

template <typename T, int NT, int G, int R>
__global__ void __launch_bounds__(NT, 1) k_cpqr_reg(const CpqrTask<T>* __restrict__ tasks,
                                                      const int32_t* __restrict__ list,
                                                      const CpqrNbr<T>* __restrict__ nbrs,
                                                      int32_t* __restrict__ cur_size, T eps) {
  typedef typename CqVec<T>::t V;
  typedef CqrShape<T, G, R> S;
  constexpr int VW = S::VW, RS = S::RS, SL = S::SL, NCH = S::NCH;
  constexpr int NW = NT / 32;
  constexpr int NGRP = NT / G;  // columns per CTA
  static_assert(R % 8 == 0 && 32 % G == 0, "slot chunks of 8, groups within a warp");
  static_assert(((RS * (int)sizeof(T) / 16) & 1) == 1, "odd 16-byte segment stride");
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const CpqrTask<T> d = tasks[list[blockIdx.x / C]];
  const int np = d.np;
  const int L = cq_ld<T>(np);
  const int nnb = d.nend - d.nbeg;
  const int npp = np > 0 ? np : 1;
  const int cpm = d.m_max > 0 ? (d.m_max + C - 1) / C : 1;
  extern __shared__ __align__(16) unsigned char smraw[];
  size_t off = cq_al16(sizeof(CqShared<T>));  // (unused here: keeps the fixed layout of the chunked kernel)
  CpqrNbr<T>* nbr = reinterpret_cast<CpqrNbr<T>*>(smraw + off);
  off += cq_al16((size_t)nnb * sizeof(CpqrNbr<T>));
  int* cstart = reinterpret_cast<int*>(smraw + off);
  off += cq_al16((size_t)(nnb + 1) * sizeof(int));
  T* tau_s = reinterpret_cast<T*>(smraw + off);  // alpha_k during the steps, tau_k after
  off += cq_al16((size_t)npp * sizeof(T));
  T* beta_s = reinterpret_cast<T*>(smraw + off);
  off += cq_al16((size_t)npp * sizeof(T));
  T* scal_s = reinterpret_cast<T*>(smraw + off);
  off += cq_al16((size_t)npp * sizeof(T));
  int* piv_s = reinterpret_cast<int*>(smraw + off);
  off += cq_al16((size_t)npp * sizeof(int));
  int* tcol = reinterpret_cast<int*>(smraw + off);
  off += cq_al16((size_t)3 * cpm * sizeof(int));
  CqrShared<T>& sh = *reinterpret_cast<CqrShared<T>*>(smraw + off);
  off += cq_al16(sizeof(CqrShared<T>));
  T* uni = reinterpret_cast<T*>(smraw + off);  // staging chunk, or the pivot slots
  T* const wslot = uni;                        // [parity][warp][SL]
  T* const cbuf = uni + (size_t)2 * NW * SL;   // [parity][source CTA][SL]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

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
    return;
  }
  const int cols_per = (m + C - 1) / C;
  if (cols_per > NGRP || np > G * R) {  // the host sizes the launch so that this never holds
    if (rank == 0 && tid == 0) cq_rank_dst(d, cur_size)[d.p] = -1;
    return;  // uniform across the cluster
  }
  const int j0 = min(m, rank * cols_per);
  const int nc = min(m, j0 + cols_per) - j0;
  T* const chunk = uni;
  int* rstep = tcol + 2 * cpm;
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
  const int cbe = ((np + G - 1) / G + 7) >> 3;  // chunks that hold rows < np
  const int kmax = min(np, m);
  // bytes a CTA receives at step k: C records and C pivot slots (live chunks)
  auto xbytes = [&](int k) -> unsigned {
    return (unsigned)C * (unsigned)(G * (cbe - k / (8 * G)) * 8 * (int)sizeof(T) + (int)sizeof(CqrRec<T>));
  };
  if (C > 1 && tid == 0) {  // visible to the cluster at the barrier after the register load
    cqr_bar_init(&sh.bar[0]);
    cqr_bar_init(&sh.bar[1]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    cqr_bar_expect(&sh.bar[0], xbytes(0));
    if (kmax > 1) cqr_bar_expect(&sh.bar[1], xbytes(1));
  }
  __syncthreads();
  bool timed_out = false;
  // ---- gather my columns of A_pn into the staging chunk (8 columns per warp
  // pass, lanes over rows, all loads before the stores)
  constexpr int GU = 8;
  for (int jb = warp * GU; jb < nc; jb += NW * GU) {
    const T* src[GU];
#pragma unroll
    for (int u = 0; u < GU; ++u) src[u] = d.Rp + (size_t)tcol[cpm + min(jb + u, nc - 1)] * d.ldp;
    for (int i = lane; i < np; i += 32) {
      T v[GU];
#pragma unroll
      for (int u = 0; u < GU; ++u) v[u] = (jb + u < nc) ? src[u][i] : T(0);
#pragma unroll
      for (int u = 0; u < GU; ++u)
        if (jb + u < nc) chunk[(size_t)(jb + u) * L + i] = v[u];
    }
  }
  __syncthreads();
  // ---- my column into registers, its squared norm
  const int grp = tid / G, g = tid % G;
  const bool own = grp < nc;
  const int gbase = lane & ~(G - 1);
  const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << gbase);
  T x[R];
  T nrm;
  {
    T s = 0;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int i = q * G + g;
      x[q] = T(0);
      if (own && i < np) x[q] = chunk[(size_t)grp * L + i];
      s = fma(x[q], x[q], s);
    }
    s = cqr_group_sum<G>(s, gmask);
    nrm = own ? s : T(-1);
  }
  // the staging chunk becomes the pivot slots, into which the other CTAs of
  // the cluster store from step 0 on: no CTA sends before every CTA has
  // loaded its columns and armed its barriers
  if (C > 1) cluster.sync();
  else __syncthreads();

  int r = kmax;
  T r00 = T(0);
  for (int k = 0; k < kmax; ++k) {
    const int cb0 = k / (8 * G);  // first live chunk
    const int par = k & 1;
    // 1. the warp's candidate (largest trailing norm, lowest index); its group
    //    derives the reflector it would define and writes u into the warp's
    //    pivot slot (chunks below cbe; zeros above row k, alpha - beta at row k)
    const bool live = own && nrm >= T(0);
    int bj = live ? j0 + grp : INT_MAX;
    T bv = live ? nrm : T(-1);
    cq_warp_argmax(bv, bj);
    if (bj != INT_MAX && bj == j0 + grp) {
      V* sl = reinterpret_cast<V*>(wslot + ((size_t)par * NW + warp) * SL + g * RS);
#pragma unroll
      for (int c = 0; c < NCH; ++c)
        if (c > cb0 && c < cbe) {
#pragma unroll
          for (int u = 0; u < 8; u += VW) {
            V v;
            if constexpr (VW == 4) v = make_float4(x[c * 8 + u], x[c * 8 + u + 1], x[c * 8 + u + 2], x[c * 8 + u + 3]);
            else v = make_double2(x[c * 8 + u], x[c * 8 + u + 1]);
            sl[(c * 8 + u) / VW] = v;
          }
        }
      cqr_chunk<NCH>(cb0, [&](auto cc) {
        constexpr int c = decltype(cc)::value;
        const int qk = k / G;
        T a = T(0);
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (c * 8 + u == qk) a = x[c * 8 + u];
        a = __shfl_sync(gmask, a, gbase + (k - qk * G));
        const T rkk = sqrt(bv);
        const T b = a >= T(0) ? -rkk : rkk;
        const T gam = rkk == T(0) ? T(0) : T(1) / (b * (b - a));
        const T amb = a - b;
        T y[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int i = (c * 8 + u) * G + g;
          y[u] = i < k ? T(0) : (i == k ? amb : x[c * 8 + u]);
        }
#pragma unroll
        for (int u = 0; u < 8; u += VW) {
          V v;
          if constexpr (VW == 4) v = make_float4(y[u], y[u + 1], y[u + 2], y[u + 3]);
          else v = make_double2(y[u], y[u + 1]);
          sl[(c * 8 + u) / VW] = v;
        }
        if (g == 0) sh.w[par][warp] = CqrRec<T>{bv, a, b, gam, bj, 0};
      });
    }
    if (bj == INT_MAX && lane == 0) sh.w[par][warp] = CqrRec<T>{T(-1), T(0), T(0), T(0), INT_MAX, 0};
    __syncthreads();
    // 2. pivot (identical in every thread of the cluster) and its reflector
    T gv = lane < NW ? sh.w[par][lane].v : T(-1);
    int gj = lane < NW ? sh.w[par][lane].j : INT_MAX;
    cq_warp_argmax(gv, gj);
    const int ww = gj == INT_MAX ? 0 : ((gj - j0) * G) >> 5;  // warp of the CTA's winner
    const T* pslot;
    CqrRec<T> rec;
    if (C == 1) {
      pslot = wslot + ((size_t)par * NW + ww) * SL;
      rec = sh.w[par][ww];
    } else {
      constexpr int SV = RS / VW;  // vectors per lane segment
      const unsigned lbar = cqr_smem_addr(&sh.bar[par]);
      if (tid < G * SV) {  // the CTA's winning slot (any slot when it has none), live vectors, into every CTA
        const int vv = tid % SV;
        if (vv >= cb0 * (8 / VW) && vv < cbe * (8 / VW)) {
          const uint4 v = reinterpret_cast<const uint4*>(wslot + ((size_t)par * NW + ww) * SL)[tid];
          const unsigned la = cqr_smem_addr(reinterpret_cast<const uint4*>(cbuf + ((size_t)par * C + rank) * SL) + tid);
          for (int q = 0; q < C; ++q) cqr_st_async(cqr_mapa(la, q), v, cqr_mapa(lbar, q));
        }
      }
      if (warp == 0 && lane < C) {
        CqrRec<T> w = sh.w[par][ww];
        if (gj == INT_MAX) w.v = T(-1), w.j = INT_MAX;
        const unsigned la = cqr_smem_addr(&sh.c[par][rank]), rb = cqr_mapa(lbar, lane);
        const uint4* wv = reinterpret_cast<const uint4*>(&w);
#pragma unroll
        for (int e = 0; e < (int)(sizeof(CqrRec<T>) / 16); ++e) cqr_st_async(cqr_mapa(la + 16 * e, lane), wv[e], rb);
      }
      // one thread waits (bounded) for the C records and slots of step k; the
      // block barrier hands the data and the outcome to the CTA
      bool late = false;
      if (tid == 0) {
        late = !cqr_bar_wait(&sh.bar[par], (unsigned)(k >> 1) & 1u);
        if (!late && k + 2 < kmax) cqr_bar_expect(&sh.bar[par], xbytes(k + 2));
      }
      if (__syncthreads_or(late)) {
        timed_out = true;
        r = k;
        break;
      }
      gv = lane < C ? sh.c[par][lane].v : T(-1);
      gj = lane < C ? sh.c[par][lane].j : INT_MAX;
      const int cj = gj;
      cq_warp_argmax(gv, gj);
      const unsigned hit = __ballot_sync(0xffffffffu, lane < C && cj == gj);
      const int owner = hit ? __ffs(hit) - 1 : 0;
      pslot = cbuf + ((size_t)par * C + owner) * SL;
      rec = sh.c[par][owner];
    }
    if (gj == INT_MAX) gj = 0;  // unreachable: k < kmax <= m leaves a live column
    const T rkk = fabs(rec.b);
    if (k == 0) r00 = rkk;
    if (r00 == T(0) || rkk < eps * r00) {
      r = k;
      break;
    }
    const bool upd = live && j0 + grp != gj;  // the pivot column leaves the live set
    if (tid == 0) {
      tau_s[k] = rec.a;
      beta_s[k] = rec.b;
      piv_s[k] = gj;
      if (gj >= j0 && gj < j0 + nc) rstep[gj - j0] = k;
    }
    // 3. H_k = I - gam u u^T on my live column (every lane runs it: a zero
    //    factor leaves retired and absent columns unchanged), then the
    //    squared norm of its rows > k
    {
      const T* ps = pslot + g * RS;
      auto ld8 = [&](int c, T (&p)[8]) {
#pragma unroll
        for (int u = 0; u < 8; u += VW) {
          const V v = reinterpret_cast<const V*>(ps + c * 8)[u / VW];
          p[u] = v.x;
          p[u + 1] = v.y;
          if constexpr (VW == 4) {
            p[u + 2] = v.z;
            p[u + 3] = v.w;
          }
        }
      };
      T a0 = 0, a1 = 0;
      cqr_chunks<NCH>(cb0, cbe, [&](auto cc) {
        constexpr int c = decltype(cc)::value;
        T p[8];
        ld8(c, p);
#pragma unroll
        for (int u = 0; u < 8; u += 2) {
          a0 = fma(x[c * 8 + u], p[u], a0);
          a1 = fma(x[c * 8 + u + 1], p[u + 1], a1);
        }
      });
      const T dot = cqr_group_sum<G>(a0 + a1, 0xffffffffu);
      const T ws = upd ? rec.gam * dot : T(0);
      T q0 = 0, q1 = 0;
      cqr_chunk<NCH>(cb0, [&](auto cc) {
        constexpr int c = decltype(cc)::value;
        T p[8];
        ld8(c, p);
#pragma unroll
        for (int u = 0; u < 8; u += 2) {
          x[c * 8 + u] = fma(-ws, p[u], x[c * 8 + u]);
          x[c * 8 + u + 1] = fma(-ws, p[u + 1], x[c * 8 + u + 1]);
          const int i = (c * 8 + u) * G + g;
          if (i > k) q0 = fma(x[c * 8 + u], x[c * 8 + u], q0);
          if (i + G > k) q1 = fma(x[c * 8 + u + 1], x[c * 8 + u + 1], q1);
        }
      });
      cqr_chunks<NCH>(cb0 + 1, cbe, [&](auto cc) {
        constexpr int c = decltype(cc)::value;
        T p[8];
        ld8(c, p);
#pragma unroll
        for (int u = 0; u < 8; u += 2) {
          x[c * 8 + u] = fma(-ws, p[u], x[c * 8 + u]);
          x[c * 8 + u + 1] = fma(-ws, p[u + 1], x[c * 8 + u + 1]);
          q0 = fma(x[c * 8 + u], x[c * 8 + u], q0);
          q1 = fma(x[c * 8 + u + 1], x[c * 8 + u + 1], q1);
        }
      });
      const T q = cqr_group_sum<G>(q0 + q1, 0xffffffffu);
      nrm = upd ? q : T(-1);
    }
  }
  __syncthreads();  // the pivot slots become the staging chunk
  for (int kk = tid; kk < r; kk += NT) {  // tau_k and scal_k from alpha_k and beta_k
    const T a = tau_s[kk], b = beta_s[kk];
    tau_s[kk] = b == T(0) ? T(0) : (b - a) / b;
    scal_s[kk] = b == T(0) ? T(0) : T(1) / (a - b);
  }
  if (own) {
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int i = q * G + g;
      if (i < np) chunk[(size_t)grp * L + i] = x[q];
    }
  }
  __syncthreads();
  cq_finish<T, NT>(d, cluster, C, rank, chunk, L, np, r, nc, j0, cpm, tcol, rstep, beta_s, scal_s, tau_s, piv_s,
                   nbr, cstart, cur_size);
  // after the epilogue's last cluster barrier, so that it follows rank 0's
  // store of the rank
  if (timed_out && threadIdx.x == 0) cq_rank_dst(d, cur_size)[d.p] = -2;
}

}  // namespace spand

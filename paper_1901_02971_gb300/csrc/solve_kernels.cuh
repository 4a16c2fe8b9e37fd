// Preconditioner apply z = M M^T r (Sec. 2.8) and the PCG vector kernels.
//
// M is the product of the elementary transforms recorded by the
// factorization.  The forward sweep (leaf -> root) applies, per step,
//   E_s: r_s <- U_s^{-T} r_s, r_n <- r_n - X_ns r_s        (Sec. 2.4)
//   S_p: r_p <- U_p^{-T} r_p                               (Sec. 2.5)
//   Q_p^T: c <- Q_pc^T r_p, fine part left in place        (Sec. 2.6.1)
// or, for the interpolative variants (Sec. 2.6.2), T_p^T: r_f <- r_f -
// T_cf^T r_c followed by the elimination of f, both elimination ops (the
// first with U = I and X^T = T_cf),
// and the backward sweep (root -> leaf) the transposes in reverse order.  The
// sparsification transform is kept as the explicit coarse basis Q_pc: since
// the fine dofs are identity in M^T A M, Q_p [c; f] = r_p + Q_pc (c - c_old)
// with r_p the forward input, so only Q_pc (|p| x r) and the forward input
// (saved per apply) are needed.  Triangular solves with the pivot factors use
// their explicit inverses Y = U^{-T} (formed once by the factorization), so
// every step of the apply is a set of independent, coalesced GEMVs.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace spand {

constexpr int AT = 256;  // threads per CTA of the apply kernels

template <typename TF>
struct ElimOp {
  const TF* XT;      // X^T, ns x m, leading dimension ld >= ns (the right part of s's
                     // block row [U_s | X^T]; T_cf for an interpolation transform)
  const TF* Y;       // U_s^{-T} (lower, ns x ns, ld = ns); nullptr: U_s = I (the
                     // interpolation transform T_p of Sec. 2.6.2)
  int32_t ns, m, ld, pad;
  int64_t slot;      // ns slots of s, then m slots of the neighbour columns
  int64_t ty, tu, ta;  // temp offsets: y_s (ns), u = X_ns y_s (m), backward acc (ns)
};

struct ApplyItem {   // one CTA's share of an operation: op index and first row / column
  int32_t op, first;
};

template <typename TF>
struct SqOp {        // scaling S_p followed (if p is sparsified) by Q_p^T, one cluster
  const TF* Y;       // U_p^{-T} (lower, np x np, ld = np)
  const TF* Q;       // coarse basis Q_pc (np x r, ld = np); nullptr: not sparsified (r = np)
  int32_t np, r;
  int64_t slot;      // np slots of p
  int64_t save;      // np (scaled forward input) + r (coarse values) entries, kept per apply
  int64_t tz;        // temp: np entries of the backward sweep
};

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------- forward sweep

constexpr int RB = 32;       // rows per item of the row-block GEMVs (one per lane)
constexpr int AP_COLS = 32;  // columns per item of the column-dot GEMVs (four per warp)
constexpr int SCH = 2048;    // input-vector chunk staged in shared memory (elements)

// Vectors written during the apply by other CTAs are read through L2 (ld.cg):
// the L1 of an SM is not coherent with writes made by other SMs.
__device__ __forceinline__ double ldv(const double* p) { return __ldcg(p); }

// Row-block GEMV: out[r] = sum_{k < K} A[r + k*ld] v(k) for the 32 rows
// r = r0 + lane, with v staged in shared memory in chunks of SCH and the
// chunk's columns split over the 8 warps (lanes cover consecutive rows, so
// every load is one coalesced 32-element segment; eight loads in flight per
// thread).  Partial sums are combined in a fixed order.  All threads call it;
// the result is valid in warp 0.
template <typename TF, typename ACC, typename Src>
__device__ __forceinline__ ACC rowblock_gemv(const TF* __restrict__ A, size_t ld, int r0, int nrows, int K, Src src,
                                             ACC* vs, ACC (*part)[RB + 1]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = AT / 32;
  const int row = r0 + lane;
  const bool live = row < nrows;
  ACC s0 = 0, s1 = 0, s2 = 0, s3 = 0;
  for (int k0 = 0; k0 < K; k0 += SCH) {
    const int kn = min(SCH, K - k0);
    __syncthreads();  // the previous chunk has been consumed
    for (int k = threadIdx.x; k < kn; k += AT) vs[k] = (ACC)src(k0 + k);
    __syncthreads();
    const int kc = (kn + nw - 1) / nw;
    const int kb = min(kn, warp * kc), ke = min(kn, kb + kc);
    if (live) {
      const TF* ap = A + row + (size_t)(k0 + kb) * ld;
      int k = kb;
      for (; k + 8 <= ke; k += 8) {
        TF a[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) a[u] = __ldg(ap + (size_t)u * ld);
        s0 = fma((ACC)a[0], vs[k], s0);
        s1 = fma((ACC)a[1], vs[k + 1], s1);
        s2 = fma((ACC)a[2], vs[k + 2], s2);
        s3 = fma((ACC)a[3], vs[k + 3], s3);
        s0 = fma((ACC)a[4], vs[k + 4], s0);
        s1 = fma((ACC)a[5], vs[k + 5], s1);
        s2 = fma((ACC)a[6], vs[k + 6], s2);
        s3 = fma((ACC)a[7], vs[k + 7], s3);
        ap += 8 * ld;
      }
      for (; k < ke; ++k, ap += ld) s0 = fma((ACC)__ldg(ap), vs[k], s0);
    }
  }
  part[warp][lane] = (s0 + s1) + (s2 + s3);
  __syncthreads();
  ACC t = 0;
  if (warp == 0)
    for (int w = 0; w < nw; ++w) t += part[w][lane];
  __syncthreads();
  return t;
}

template <typename ACC>
__device__ __forceinline__ ACC warp_sum(ACC v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Column-dot GEMV: out(j) = sum_{i in [lo_j, n)} A[i + j*ld] v(i) for the
// columns j in [c0, c1) (at most AP_COLS), lo_j = j if `tri` (A lower
// triangular: rows above the diagonal are never read) else 0.  Warp w owns
// columns c0 + w + 8q (q < 4) and sweeps them together, lanes over i, so four
// to eight loads are in flight per lane; v is staged in chunks of SCH.  All
// threads call it; `store(j, value)` runs on lane 0 of the owning warp.
template <typename TF, typename ACC, typename Src, typename Store>
__device__ __forceinline__ void coldot_gemv(const TF* __restrict__ A, size_t ld, int n, int c0, int c1, bool tri,
                                            Src src, Store store, ACC* vs) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = AT / 32;
  int j[4];
  bool ok[4];
  ACC acc[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    j[q] = c0 + warp + nw * q;
    ok[q] = j[q] < c1;
    acc[q] = 0;
  }
  const int lo = tri ? c0 : 0;  // no column of this item reads rows above c0
  for (int i0 = lo; i0 < n; i0 += SCH) {
    const int in = min(SCH, n - i0);
    __syncthreads();
    for (int i = threadIdx.x; i < in; i += AT) vs[i] = (ACC)src(i0 + i);
    __syncthreads();
    int i = lane;
    for (; i + 32 < in; i += 64) {
      TF a[4][2];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const TF* col = A + (size_t)j[q] * ld + i0;
        const bool t0 = ok[q] && (!tri || i0 + i >= j[q]);
        const bool t1 = ok[q] && (!tri || i0 + i + 32 >= j[q]);
        a[q][0] = t0 ? __ldg(col + i) : TF(0);
        a[q][1] = t1 ? __ldg(col + i + 32) : TF(0);
      }
      const ACC v0 = vs[i], v1 = vs[i + 32];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = fma((ACC)a[q][1], v1, fma((ACC)a[q][0], v0, acc[q]));
    }
    for (; i < in; i += 32) {
      const ACC v0 = vs[i];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (ok[q] && (!tri || i0 + i >= j[q])) acc[q] = fma((ACC)__ldg(A + (size_t)j[q] * ld + i0 + i), v0, acc[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const ACC v = warp_sum(acc[q]);
    if (ok[q] && lane == 0) store(j[q], v);
  }
}

// ---------------------------------------------------------------- the persistent apply
//
// The whole apply is one cooperative launch that walks the phases of every
// step in order (forward: leaves -> root, backward: root -> leaves) with a
// grid-wide barrier between dependent phases; within a phase the items are
// independent and are spread over all CTAs.

enum ApplyKind : int32_t {
  PH_FY = 0,   // E_s forward:  y_s = Y x_s                  -> tmp[ty]
  PH_FU,       //               u = X_ns y_s                  -> tmp[tu]
  PH_SCATTER,  //               x_s = y_s, x_n -= sum u (pull, fixed order)
  PH_SY,       // S_p forward:  y_p = Y x_p                  -> save[0:np]
  PH_SC,       // Q_p^T:        c = Q_pc^T y_p               -> x (coarse slots), save[np:np+r]
  PH_SZ,       // Q_p backward: z = y_p + Q_pc (c - c_old)   -> tmp[tz]
  PH_SX,       // S_p backward: x_p = Y^T z
  PH_BA,       // E_s backward: acc = x_s - X_ns^T x_n       -> tmp[ta]
  PH_BX        //               x_s = Y^T acc
};

template <typename TF>
struct __align__(8) ApplyPhase {
  int32_t kind, n;             // n = items, or scatter targets
  const ElimOp<TF>* elim;
  const SqOp<TF>* sq;
  const ApplyItem* items;
  const int32_t* slots;
  const int32_t* tslot;        // scatter only
  const int64_t* tptr;
  const int64_t* tidx;
  int64_t nassign;
};
static_assert(sizeof(ApplyPhase<float>) % 8 == 0 && sizeof(ApplyPhase<double>) % 8 == 0, "phase table copy");

constexpr unsigned kBarrierSpins = 1u << 24;  // with ~40 ns sleeps: well over a second

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier on a monotonically increasing arrival counter (reset to 0
// before the launch): barrier b completes when the counter reaches
// (b + 1) * gridDim.x.  All CTAs are co-resident (cooperative launch).  The
// CTA's writes are ordered before its arrival by bar.sync + a release fence,
// and the waiter's acquire load + fence order the next phase's reads after
// every arrival.  The wait is bounded: on timeout *err is set and false is
// returned to every thread of the CTA, which then leaves the kernel.
__device__ __forceinline__ void grid_arrive(unsigned* count) {
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    asm volatile("red.relaxed.gpu.global.add.u32 [%0], %1;" ::"l"(count), "r"(1u) : "memory");
  }
}

__device__ __forceinline__ bool grid_wait(const unsigned* count, unsigned target, int* err, unsigned limit) {
  __shared__ int ok;
  if (threadIdx.x == 0) {
    ok = 1;
    unsigned spins = 0;
    while (ld_acquire_u32(count) < target) {
      if (++spins > limit) {
        atomicExch(err, 1);
        ok = 0;
        break;
      }
      if (spins > 64) __nanosleep(32);
    }
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
  }
  __syncthreads();
  return ok != 0;
}

__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// Warm the caches for this CTA's first item of phase P (read-only data only:
// the item, its op, its slot list, and the lines of the factor block it
// streams).  Runs between arriving at a grid barrier and waiting on it.
template <typename TF>
__device__ __forceinline__ void prefetch_first_item(const ApplyPhase<TF>& P) {
  if (P.kind == PH_SCATTER || (int)blockIdx.x >= P.n) return;
  const ApplyItem it = P.items[blockIdx.x];
  const TF* A;
  size_t ld;
  int rows, lo, cols;     // row-block items: 32 rows from `lo`, `cols` columns; column items: `cols` from `lo`
  bool rowblock;
  const int32_t* sl;
  int nsl;
  if (P.kind == PH_FY || P.kind == PH_BA || P.kind == PH_FU || P.kind == PH_BX) {
    const ElimOp<TF> o = P.elim[it.op];
    sl = P.slots + o.slot;
    ld = (size_t)o.ns;
    rows = o.ns;
    if (P.kind == PH_FY) { A = o.Y; rowblock = true; lo = it.first; cols = min(o.ns, it.first + RB); nsl = cols; }
    else if (P.kind == PH_BA) { A = o.XT; ld = (size_t)o.ld; rowblock = true; lo = it.first; cols = o.m; sl += o.ns; nsl = o.m; }
    else if (P.kind == PH_FU) { A = o.XT; ld = (size_t)o.ld; rowblock = false; lo = it.first; cols = min(o.m - it.first, AP_COLS); nsl = 0; }
    else { A = o.Y; rowblock = false; lo = it.first; cols = min(o.ns - it.first, AP_COLS); nsl = cols + it.first; }
  } else {
    const SqOp<TF> o = P.sq[it.op];
    sl = P.slots + o.slot;
    ld = (size_t)o.np;
    rows = o.np;
    if (P.kind == PH_SY) { A = o.Y; rowblock = true; lo = it.first; cols = min(o.np, it.first + RB); nsl = cols; }
    else if (P.kind == PH_SZ) { A = o.Q; rowblock = true; lo = it.first; cols = o.Q ? o.r : 0; nsl = o.r; }
    else if (P.kind == PH_SC) { A = o.Q; rowblock = false; lo = it.first; cols = o.Q ? min(o.r - it.first, AP_COLS) : 0; nsl = 0; }
    else { A = o.Y; rowblock = false; lo = it.first; cols = min(o.np - it.first, AP_COLS); nsl = o.np; }
  }
  for (int k = threadIdx.x * 32; k < nsl; k += AT * 32) prefetch_l2(sl + k);
  if (!A || cols <= 0) return;
  if (rowblock) {
    for (int k = threadIdx.x; k < cols; k += AT) prefetch_l2(A + lo + (size_t)k * ld);
  } else {  // columns lo .. lo+cols-1, contiguous: one line per 128 bytes
    const char* b = reinterpret_cast<const char*>(A + (size_t)lo * ld);
    const size_t bytes = (size_t)cols * ld * sizeof(TF);
    for (size_t off = (size_t)threadIdx.x * 128; off < bytes; off += (size_t)AT * 128) prefetch_l2(b + off);
  }
  (void)rows;
}

// spin_limit bounds every barrier wait (kBarrierSpins by default); bias is
// added to every barrier target (0 in normal use; a failure-path test sets 1,
// a target no arrival count reaches, so that every wait runs out).
template <typename TF>
__global__ void __launch_bounds__(AT) k_apply(const ApplyPhase<TF>* __restrict__ phases, int nph, double* x,
                                              double* tmp, double* save, unsigned* bar, int* err,
                                              unsigned spin_limit, unsigned bias) {
  typedef TF ACC;  // inner sums in the factor's precision
  extern __shared__ __align__(16) unsigned char apply_smem[];
  ACC* vs = reinterpret_cast<ACC*>(apply_smem);
  // the phase table, copied once (its loads are off the per-phase critical path)
  ApplyPhase<TF>* ptab = reinterpret_cast<ApplyPhase<TF>*>(apply_smem + SCH * sizeof(ACC));
  __shared__ ACC part[AT / 32][RB + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  {
    const int words = nph * (int)(sizeof(ApplyPhase<TF>) / 8);
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(phases);
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(ptab);
    for (int w = threadIdx.x; w < words; w += AT) dst[w] = src[w];
    __syncthreads();
  }
  for (int p = 0; p < nph; ++p) {
    const ApplyPhase<TF>& P = ptab[p];
    if (P.kind == PH_SCATTER) {
      for (int64_t t = blockIdx.x * (int64_t)AT + threadIdx.x; t < P.n; t += (int64_t)gridDim.x * AT) {
        if (t < P.nassign) {
          x[P.tslot[t]] = ldv(tmp + P.tidx[P.tptr[t]]);
        } else {
          double s = 0.0;
          for (int64_t e = P.tptr[t]; e < P.tptr[t + 1]; ++e) s += ldv(tmp + P.tidx[e]);
          x[P.tslot[t]] = ldv(x + P.tslot[t]) - s;
        }
      }
    } else {
      for (int itx = blockIdx.x; itx < P.n; itx += gridDim.x) {
        const ApplyItem it = P.items[itx];
        if (P.kind == PH_FY || P.kind == PH_BA || P.kind == PH_FU || P.kind == PH_BX) {
          const ElimOp<TF> o = P.elim[it.op];
          const int32_t* sl = P.slots + o.slot;
          const TF* XT = o.XT;
          if (P.kind == PH_FY) {
            const int i = it.first + lane;
            if (!o.Y) {
              if (warp == 0 && i < o.ns) tmp[o.ty + i] = ldv(x + sl[i]);
            } else {
              const int K = min(o.ns, it.first + RB);
              const ACC v = rowblock_gemv<TF, ACC>(o.Y, (size_t)o.ns, it.first, o.ns, K,
                                                   [&](int k) { return ldv(x + sl[k]); }, vs, part);
              if (warp == 0 && i < o.ns) tmp[o.ty + i] = (double)v;
            }
          } else if (P.kind == PH_BA) {
            const ACC v = rowblock_gemv<TF, ACC>(XT, (size_t)o.ld, it.first, o.ns, o.m,
                                                 [&](int k) { return ldv(x + sl[o.ns + k]); }, vs, part);
            const int i = it.first + lane;
            if (warp == 0 && i < o.ns) tmp[o.ta + i] = ldv(x + sl[i]) - (double)v;
          } else if (P.kind == PH_FU) {
            coldot_gemv<TF, ACC>(XT, (size_t)o.ld, o.ns, it.first, min(o.m, it.first + AP_COLS), false,
                                 [&](int i) { return ldv(tmp + o.ty + i); },
                                 [&](int j, ACC v) { tmp[o.tu + j] = (double)v; }, vs);
          } else if (!o.Y) {  // PH_BX, U_s = I
            for (int j = it.first + threadIdx.x; j < min(o.ns, it.first + AP_COLS); j += AT) x[sl[j]] = ldv(tmp + o.ta + j);
          } else {  // PH_BX
            coldot_gemv<TF, ACC>(o.Y, (size_t)o.ns, o.ns, it.first, min(o.ns, it.first + AP_COLS), true,
                                 [&](int i) { return ldv(tmp + o.ta + i); },
                                 [&](int j, ACC v) { x[sl[j]] = (double)v; }, vs);
          }
        } else {
          const SqOp<TF> o = P.sq[it.op];
          const int32_t* sl = P.slots + o.slot;
          double* sv = save + o.save;
          if (P.kind == PH_SY) {
            const int K = min(o.np, it.first + RB);
            const ACC v = rowblock_gemv<TF, ACC>(o.Y, (size_t)o.np, it.first, o.np, K,
                                                 [&](int k) { return ldv(x + sl[k]); }, vs, part);
            const int i = it.first + lane;
            if (warp == 0 && i < o.np) sv[i] = (double)v;
          } else if (P.kind == PH_SC) {
            const int hi = min(o.r, it.first + AP_COLS);
            if (o.Q) {
              coldot_gemv<TF, ACC>(o.Q, (size_t)o.np, o.np, it.first, hi, false, [&](int i) { return ldv(sv + i); },
                                   [&](int k, ACC c) {
                                     x[sl[k]] = (double)c;
                                     sv[o.np + k] = (double)c;
                                   },
                                   vs);
            } else {
              for (int k = it.first + threadIdx.x; k < hi; k += AT) {
                const double c = ldv(sv + k);
                x[sl[k]] = c;
                sv[o.np + k] = c;
              }
            }
          } else if (P.kind == PH_SZ) {
            const int i = it.first + lane;
            if (!o.Q) {
              if (warp == 0 && i < o.np) tmp[o.tz + i] = ldv(x + sl[i]);
            } else {
              const ACC v = rowblock_gemv<TF, ACC>(o.Q, (size_t)o.np, it.first, o.np, o.r,
                                                   [&](int k) { return ldv(x + sl[k]) - ldv(sv + o.np + k); }, vs, part);
              if (warp == 0 && i < o.np) tmp[o.tz + i] = ldv(sv + i) + (double)v;
            }
          } else {  // PH_SX
            coldot_gemv<TF, ACC>(o.Y, (size_t)o.np, o.np, it.first, min(o.np, it.first + AP_COLS), true,
                                 [&](int i) { return ldv(tmp + o.tz + i); },
                                 [&](int j, ACC v) { x[sl[j]] = (double)v; }, vs);
          }
        }
      }
    }
    if (p + 1 < nph) {
      grid_arrive(bar);
      prefetch_first_item(ptab[p + 1]);
      if (!grid_wait(bar, (unsigned)(p + 1) * gridDim.x + bias, err, spin_limit)) return;
    }
  }
}

// ---------------------------------------------------------------- PCG pieces

constexpr int RED_BLOCKS = 608;  // 4 x 152 SMs
constexpr int RED_THREADS = 256;

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sred[RED_THREADS / 32];
  v = warp_sum_d(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sred[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sred[w];
  __syncthreads();
  return s;
}

// q = A p (CSR, 4 lanes per row) and per-block partial sums of p.q
__global__ void __launch_bounds__(RED_THREADS) k_spmv_dot(int64_t n, const int64_t* __restrict__ rp,
                                                          const int32_t* __restrict__ ci, const double* __restrict__ va,
                                                          const double* __restrict__ p, double* __restrict__ q,
                                                          double* __restrict__ part) {
  const int sub = threadIdx.x & 3;
  double acc = 0.0;
  // the loop bound is uniform across a warp so that every lane reaches the shuffles
  const int64_t stride = ((int64_t)gridDim.x * blockDim.x) >> 2;
  for (int64_t base = (blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31)) >> 2; base < n; base += stride) {
    const int64_t row = base + ((threadIdx.x & 31) >> 2);
    double s = 0.0;
    if (row < n)
      for (int64_t e = rp[row] + sub; e < rp[row + 1]; e += 4) s += va[e] * p[ci[e]];
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    if (sub == 0 && row < n) {
      q[row] = s;
      acc += s * p[row];
    }
  }
  const double b = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = b;
}

// out[0] = sum(part[0:nb])  (fixed order)
__global__ void k_reduce(const double* __restrict__ part, int nb, double* __restrict__ out) {
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) s += part[i];
  s = block_sum(s);
  if (threadIdx.x == 0) *out = s;
}

// alpha = rz / pq; x += alpha p; r -= alpha q; partial sums of r.r
__global__ void __launch_bounds__(RED_THREADS) k_update_xr(int64_t n, const double* __restrict__ sc, double* __restrict__ x,
                                                           double* __restrict__ r, const double* __restrict__ p,
                                                           const double* __restrict__ q, double* __restrict__ part) {
  const double alpha = sc[0] / sc[1];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] += alpha * p[i];
    const double v = r[i] - alpha * q[i];
    r[i] = v;
    acc += v * v;
  }
  const double b = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = b;
}

__global__ void __launch_bounds__(RED_THREADS) k_dot(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                                                     double* __restrict__ part) {
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += a[i] * b[i];
  const double s = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// beta = rz_new / rz_old; p = z + beta p; then rz_old = rz_new (by thread 0 of block 0 after use is unsafe,
// so the host swaps the scalar slots instead).
__global__ void k_update_p(int64_t n, const double* __restrict__ rz_new, const double* __restrict__ rz_old,
                           const double* __restrict__ z, double* __restrict__ p) {
  const double beta = rz_new[0] / rz_old[0];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = z[i] + beta * p[i];
}

__global__ void k_copy_vec(int64_t n, const double* __restrict__ a, double* __restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) b[i] = a[i];
}

// y[i] = x[perm[i]] (gather into the cluster order) or y[perm[i]] = x[i] (scatter back)
__global__ void k_permute(int64_t n, const int32_t* __restrict__ perm, const double* __restrict__ x, double* __restrict__ y,
                          int gather) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (gather) y[i] = x[perm[i]];
    else y[perm[i]] = x[i];
  }
}

// out[k] = vals[src[k]] (values of A in the cluster order)
__global__ void k_gather_vals(int64_t nnz, const int64_t* __restrict__ src, const double* __restrict__ vals,
                              double* __restrict__ out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x)
    out[k] = vals[src[k]];
}

// dL/dA on A's pattern: out[e] = -lam[row(e)] * x[col(e)] (original CSR order)
__global__ void k_sampled_outer(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                const double* __restrict__ lam, const double* __restrict__ x, double* __restrict__ out) {
  for (int64_t row = blockIdx.x * (int64_t)(blockDim.x / 32) + (threadIdx.x >> 5); row < n;
       row += (int64_t)gridDim.x * (blockDim.x / 32)) {
    const double l = -lam[row];
    for (int64_t e = rp[row] + (threadIdx.x & 31); e < rp[row + 1]; e += 32) out[e] = l * x[ci[e]];
  }
}

// r = b - A x
__global__ void k_residual(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           const double* __restrict__ va, const double* __restrict__ x, const double* __restrict__ b,
                           double* __restrict__ r) {
  const int sub = threadIdx.x & 3;
  const int64_t stride = ((int64_t)gridDim.x * blockDim.x) >> 2;
  for (int64_t base = (blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31)) >> 2; base < n; base += stride) {
    const int64_t row = base + ((threadIdx.x & 31) >> 2);
    double s = 0.0;
    if (row < n)
      for (int64_t e = rp[row] + sub; e < rp[row + 1]; e += 4) s += va[e] * x[ci[e]];
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    if (sub == 0 && row < n) r[row] = b[row] - s;
  }
}

}  // namespace spand

// Preconditioner apply z = M M^T r (Sec. 2.8) and the PCG vector kernels.
//
// M is the product of the elementary transforms recorded by the
// factorization.  The forward sweep (leaf -> root) applies, per step,
//   E_s: r_s <- U_s^{-T} r_s, r_n <- r_n - X_ns r_s        (Sec. 2.4)
//   S_p: r_p <- U_p^{-T} r_p                               (Sec. 2.5)
//   Q_p^T: c <- Q_pc^T r_p, fine part left in place        (Sec. 2.6.1)
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
  const TF* R;       // [U_s | X^T], ns x (ns + m), ld = ns
  const TF* Y;       // U_s^{-T} (lower, ns x ns, ld = ns)
  int32_t ns, m;
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

// warp-wide sum_{i in [i0, n)} a[i] * x[i] (a contiguous), lanes over i,
// four independent accumulators (128 elements per iteration)
template <typename TF>
__device__ __forceinline__ double dot_warp(const TF* __restrict__ a, const double* x, int i0, int n) {
  const int lane = threadIdx.x & 31;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int i = i0 + lane;
  for (; i + 96 < n; i += 128) {
    s0 += (double)a[i] * x[i];
    s1 += (double)a[i + 32] * x[i + 32];
    s2 += (double)a[i + 64] * x[i + 64];
    s3 += (double)a[i + 96] * x[i + 96];
  }
  for (; i < n; i += 32) s0 += (double)a[i] * x[i];
  return warp_sum_d((s0 + s1) + (s2 + s3));
}

constexpr int RB = 32;       // rows per block of the row-dot kernels (one per lane)
constexpr int AP_COLS = 32;  // outputs per CTA of the warp-per-column kernels

// Row dots of a 32-row block: sum_{k < K} A[r0 + lane + k*ld] x[k], with the K
// range split over the CTA's 8 warps (lanes cover consecutive rows, so every
// load is coalesced) and the 8 partial sums added in a fixed order.  All
// threads must call it; the result is valid in warp 0 for row r0 + lane.
template <typename TF>
__device__ __forceinline__ double rowblock_dot(const TF* __restrict__ A, size_t ld, int r0, int nrows,
                                               const double* x, int K, double (*part)[RB + 1]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = AT / 32;
  const int row = r0 + lane;
  const int kc = (K + nw - 1) / nw;
  const int k0 = warp * kc, k1 = min(K, k0 + kc);
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  if (row < nrows) {
    const TF* a = A + row;
    int k = k0;
    for (; k + 4 <= k1; k += 4) {
      s0 += (double)a[(size_t)k * ld] * x[k];
      s1 += (double)a[(size_t)(k + 1) * ld] * x[k + 1];
      s2 += (double)a[(size_t)(k + 2) * ld] * x[k + 2];
      s3 += (double)a[(size_t)(k + 3) * ld] * x[k + 3];
    }
    for (; k < k1; ++k) s0 += (double)a[(size_t)k * ld] * x[k];
  }
  part[warp][lane] = (s0 + s1) + (s2 + s3);
  __syncthreads();
  double t = 0.0;
  if (warp == 0)
    for (int w = 0; w < nw; ++w) t += part[w][lane];
  __syncthreads();
  return t;
}

// forward, part 1: y_s = U_s^{-T} x_s = Y x_s for one 32-row block -> tmp[ty]
// (Y is exactly zero above its diagonal, so the block reads columns < r0 + 32)
template <typename TF>
__global__ void __launch_bounds__(AT) k_elim_fwd_y(const ElimOp<TF>* __restrict__ ops, const ApplyItem* __restrict__ items,
                                                  const int32_t* __restrict__ slots, const double* __restrict__ x,
                                                  double* __restrict__ tmp) {
  extern __shared__ double xs[];
  __shared__ double part[AT / 32][RB + 1];
  const ApplyItem it = items[blockIdx.x];
  const ElimOp<TF> o = ops[it.op];
  const int32_t* sl = slots + o.slot;
  const int K = min(o.ns, it.first + RB);
  for (int j = threadIdx.x; j < K; j += AT) xs[j] = x[sl[j]];
  __syncthreads();
  const double v = rowblock_dot(o.Y, (size_t)o.ns, it.first, o.ns, xs, K, part);
  const int i = it.first + (threadIdx.x & 31);
  if (threadIdx.x < 32 && i < o.ns) tmp[o.ty + i] = v;
}

// forward, part 2: u = X_ns y_s (X_ns = (X^T)^T), AP_COLS outputs per CTA -> tmp[tu]
template <typename TF>
__global__ void __launch_bounds__(AT) k_elim_fwd_u(const ElimOp<TF>* __restrict__ ops, const ApplyItem* __restrict__ items,
                                                  double* __restrict__ tmp) {
  extern __shared__ double ys[];
  const ApplyItem it = items[blockIdx.x];
  const ElimOp<TF> o = ops[it.op];
  for (int i = threadIdx.x; i < o.ns; i += AT) ys[i] = tmp[o.ty + i];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const TF* XT = o.R + (size_t)o.ns * o.ns;
  const int hi = min(o.m, it.first + AP_COLS);
  for (int j = it.first + warp; j < hi; j += AT / 32) {
    const double v = dot_warp(XT + (size_t)j * o.ns, ys, 0, o.ns);
    if (lane == 0) tmp[o.tu + j] = v;
  }
}

// forward, part 3: x_s = y_s (assign targets) and x_n -= sum of the u's aimed
// at it (pull form, fixed order).  Targets [0, nassign) are assignments with
// exactly one source.
__global__ void k_scatter(const int32_t* __restrict__ tslot, const int64_t* __restrict__ ptr,
                          const int64_t* __restrict__ idx, const double* __restrict__ tmp, double* __restrict__ x,
                          int64_t nassign, int64_t ntgt) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ntgt; t += (int64_t)gridDim.x * blockDim.x) {
    if (t < nassign) {
      x[tslot[t]] = tmp[idx[ptr[t]]];
    } else {
      double s = 0.0;
      for (int64_t e = ptr[t]; e < ptr[t + 1]; ++e) s += tmp[idx[e]];
      x[tslot[t]] -= s;
    }
  }
}



// ---------------------------------------------------------------- backward sweep



// ---------------------------------------------------------------- scaling + coarse basis

// forward, part 1: y_p = U_p^{-T} x_p = Y x_p for one 32-row block -> save[0:np]
template <typename TF>
__global__ void __launch_bounds__(AT) k_sq_fwd_y(const SqOp<TF>* __restrict__ ops, const ApplyItem* __restrict__ items,
                                                const int32_t* __restrict__ slots, const double* __restrict__ x,
                                                double* __restrict__ save) {
  extern __shared__ double xs[];
  __shared__ double part[AT / 32][RB + 1];
  const ApplyItem it = items[blockIdx.x];
  const SqOp<TF> o = ops[it.op];
  const int32_t* sl = slots + o.slot;
  const int K = min(o.np, it.first + RB);
  for (int j = threadIdx.x; j < K; j += AT) xs[j] = x[sl[j]];
  __syncthreads();
  const double v = rowblock_dot(o.Y, (size_t)o.np, it.first, o.np, xs, K, part);
  const int i = it.first + (threadIdx.x & 31);
  if (threadIdx.x < 32 && i < o.np) save[o.save + i] = v;
}

// forward, part 2: c = Q_pc^T y_p (identity when p is not sparsified), AP_COLS
// outputs per CTA -> x[first r slots] and save[np:np+r]
template <typename TF>
__global__ void __launch_bounds__(AT) k_sq_fwd_c(const SqOp<TF>* __restrict__ ops, const ApplyItem* __restrict__ items,
                                                const int32_t* __restrict__ slots, double* __restrict__ x,
                                                double* __restrict__ save) {
  extern __shared__ double ys[];
  const ApplyItem it = items[blockIdx.x];
  const SqOp<TF> o = ops[it.op];
  const int32_t* sl = slots + o.slot;
  double* sv = save + o.save;
  for (int i = threadIdx.x; i < o.np; i += AT) ys[i] = sv[i];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int hi = min(o.r, it.first + AP_COLS);
  for (int k = it.first + warp; k < hi; k += AT / 32) {
    const double c = o.Q ? dot_warp(o.Q + (size_t)k * o.np, ys, 0, o.np) : ys[k];
    if (lane == 0) {
      x[sl[k]] = c;
      sv[o.np + k] = c;
    }
  }
}

// backward, part 1: z = y_p + Q_pc (c - c_old) for one 32-row block -> tmp[tz]
// (without Q: z = x_p)
template <typename TF>
__global__ void __launch_bounds__(AT) k_sq_bwd_z(const SqOp<TF>* __restrict__ ops, const ApplyItem* __restrict__ items,
                                                const int32_t* __restrict__ slots, const double* __restrict__ x,
                                                const double* __restrict__ save, double* __restrict__ tmp) {
  extern __shared__ double dc[];
  __shared__ double part[AT / 32][RB + 1];
  const ApplyItem it = items[blockIdx.x];
  const SqOp<TF> o = ops[it.op];
  const int32_t* sl = slots + o.slot;
  const double* sv = save + o.save;
  const int i = it.first + (threadIdx.x & 31);
  if (!o.Q) {
    if (threadIdx.x < 32 && i < o.np) tmp[o.tz + i] = x[sl[i]];
    return;
  }
  for (int k = threadIdx.x; k < o.r; k += AT) dc[k] = x[sl[k]] - sv[o.np + k];
  __syncthreads();
  const double v = rowblock_dot(o.Q, (size_t)o.np, it.first, o.np, dc, o.r, part);
  if (threadIdx.x < 32 && i < o.np) tmp[o.tz + i] = sv[i] + v;
}

// backward, part 2: x_p = U_p^{-1} z = Y^T z, AP_COLS outputs per CTA
template <typename TF>
__global__ void __launch_bounds__(AT) k_sq_bwd_x(const SqOp<TF>* __restrict__ ops, const ApplyItem* __restrict__ items,
                                                const int32_t* __restrict__ slots, const double* __restrict__ tmp,
                                                double* __restrict__ x) {
  extern __shared__ double zs[];
  const ApplyItem it = items[blockIdx.x];
  const SqOp<TF> o = ops[it.op];
  const int32_t* sl = slots + o.slot;
  for (int i = threadIdx.x; i < o.np; i += AT) zs[i] = tmp[o.tz + i];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int hi = min(o.np, it.first + AP_COLS);
  for (int j = it.first + warp; j < hi; j += AT / 32) {
    const double v = dot_warp(o.Y + (size_t)j * o.np, zs, j, o.np);
    if (lane == 0) x[sl[j]] = v;
  }
}

// backward, part 1: acc = x_s - X_ns^T x_n for one 32-row block -> tmp[ta]
template <typename TF>
__global__ void __launch_bounds__(AT) k_elim_bwd_acc(const ElimOp<TF>* __restrict__ ops, const ApplyItem* __restrict__ items,
                                                    const int32_t* __restrict__ slots, const double* __restrict__ x,
                                                    double* __restrict__ tmp) {
  extern __shared__ double xn[];
  __shared__ double part[AT / 32][RB + 1];
  const ApplyItem it = items[blockIdx.x];
  const ElimOp<TF> o = ops[it.op];
  const int32_t* sl = slots + o.slot;
  for (int j = threadIdx.x; j < o.m; j += AT) xn[j] = x[sl[o.ns + j]];
  __syncthreads();
  const TF* XT = o.R + (size_t)o.ns * o.ns;
  const double v = rowblock_dot(XT, (size_t)o.ns, it.first, o.ns, xn, o.m, part);
  const int i = it.first + (threadIdx.x & 31);
  if (threadIdx.x < 32 && i < o.ns) tmp[o.ta + i] = x[sl[i]] - v;
}

// backward, part 2: x_s = U_s^{-1} acc = Y^T acc, AP_COLS outputs per CTA
template <typename TF>
__global__ void __launch_bounds__(AT) k_elim_bwd_x(const ElimOp<TF>* __restrict__ ops, const ApplyItem* __restrict__ items,
                                                  const int32_t* __restrict__ slots, const double* __restrict__ tmp,
                                                  double* __restrict__ x) {
  extern __shared__ double acc[];
  const ApplyItem it = items[blockIdx.x];
  const ElimOp<TF> o = ops[it.op];
  const int32_t* sl = slots + o.slot;
  for (int i = threadIdx.x; i < o.ns; i += AT) acc[i] = tmp[o.ta + i];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int hi = min(o.ns, it.first + AP_COLS);
  for (int j = it.first + warp; j < hi; j += AT / 32) {
    const double v = dot_warp(o.Y + (size_t)j * o.ns, acc, j, o.ns);
    if (lane == 0) x[sl[j]] = v;
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

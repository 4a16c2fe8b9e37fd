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
  int64_t tmp;       // m entries of the forward update
};

template <typename TF>
struct ScaleOp {
  const TF* Y;       // U_p^{-T} (lower, np x np, ld = np)
  int32_t np, pad;
  int64_t slot;
};

template <typename TF>
struct QOp {
  const TF* Q;       // np x r coarse basis, ld = np
  int32_t np, r;
  int64_t slot;
  int64_t save;      // np (forward input) + r (coarse values) entries
};

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// y = Y x, Y lower n x n (ld n): one thread per row (coalesced over rows).
template <typename TF>
__device__ __forceinline__ void trmv_lower_cta(const TF* __restrict__ Y, int n, const double* x, double* y) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double s = 0.0;
    for (int j = 0; j <= i; ++j) s += (double)Y[i + (size_t)j * n] * x[j];
    y[i] = s;
  }
}

// y_j = sum_{i >= j} Y[i, j] x_i  (y = Y^T x): one warp per output.
template <typename TF>
__device__ __forceinline__ void trmv_lowerT_warp(const TF* __restrict__ Y, int n, const double* x, int j, double& out) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int i = j + lane; i < n; i += 32) s += (double)Y[i + (size_t)j * n] * x[i];
  out = warp_sum_d(s);
}

// ---------------------------------------------------------------- forward sweep

template <typename TF>
__global__ void __launch_bounds__(AT) k_elim_fwd(const ElimOp<TF>* __restrict__ ops, const int32_t* __restrict__ slots,
                                                double* __restrict__ x, double* __restrict__ tmp) {
  extern __shared__ double sh[];
  const ElimOp<TF> o = ops[blockIdx.x];
  const int32_t* sl = slots + o.slot;
  double* xs = sh;
  double* ys = sh + o.ns;
  for (int i = threadIdx.x; i < o.ns; i += blockDim.x) xs[i] = x[sl[i]];
  __syncthreads();
  trmv_lower_cta(o.Y, o.ns, xs, ys);  // y_s = U_s^{-T} x_s
  __syncthreads();
  for (int i = threadIdx.x; i < o.ns; i += blockDim.x) x[sl[i]] = ys[i];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const TF* XT = o.R + (size_t)o.ns * o.ns;
  for (int j = warp; j < o.m; j += nw) {  // u = X_ns y_s
    double s = 0.0;
    for (int i = lane; i < o.ns; i += 32) s += (double)XT[i + (size_t)j * o.ns] * ys[i];
    s = warp_sum_d(s);
    if (lane == 0) tmp[o.tmp + j] = s;
  }
}

// x[slot_t] -= sum of the forward updates aimed at it (fixed order).
__global__ void k_scatter_sub(const int32_t* __restrict__ tslot, const int64_t* __restrict__ ptr,
                              const int64_t* __restrict__ idx, const double* __restrict__ tmp,
                              double* __restrict__ x, int64_t ntgt) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ntgt; t += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int64_t e = ptr[t]; e < ptr[t + 1]; ++e) s += tmp[idx[e]];
    x[tslot[t]] -= s;
  }
}

template <typename TF>
__global__ void __launch_bounds__(AT) k_scale_fwd(const ScaleOp<TF>* __restrict__ ops, const int32_t* __restrict__ slots,
                                                 double* __restrict__ x) {
  extern __shared__ double xs[];
  const ScaleOp<TF> o = ops[blockIdx.x];
  const int32_t* sl = slots + o.slot;
  for (int i = threadIdx.x; i < o.np; i += blockDim.x) xs[i] = x[sl[i]];
  __syncthreads();
  for (int i = threadIdx.x; i < o.np; i += blockDim.x) {  // x_p <- U_p^{-T} x_p
    double s = 0.0;
    for (int j = 0; j <= i; ++j) s += (double)o.Y[i + (size_t)j * o.np] * xs[j];
    x[sl[i]] = s;
  }
}

template <typename TF>
__global__ void __launch_bounds__(AT) k_q_fwd(const QOp<TF>* __restrict__ ops, const int32_t* __restrict__ slots,
                                             double* __restrict__ x, double* __restrict__ save) {
  extern __shared__ double ys[];
  const QOp<TF> o = ops[blockIdx.x];
  const int32_t* sl = slots + o.slot;
  double* sv = save + o.save;
  for (int i = threadIdx.x; i < o.np; i += blockDim.x) {
    const double v = x[sl[i]];
    ys[i] = v;
    sv[i] = v;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int k = warp; k < o.r; k += nw) {
    double s = 0.0;
    for (int i = lane; i < o.np; i += 32) s += (double)o.Q[i + (size_t)k * o.np] * ys[i];
    s = warp_sum_d(s);
    if (lane == 0) {
      sv[o.np + k] = s;
      x[sl[k]] = s;
    }
  }
}

// ---------------------------------------------------------------- backward sweep

template <typename TF>
__global__ void __launch_bounds__(AT) k_q_bwd(const QOp<TF>* __restrict__ ops, const int32_t* __restrict__ slots,
                                             double* __restrict__ x, const double* __restrict__ save) {
  extern __shared__ double dc[];
  const QOp<TF> o = ops[blockIdx.x];
  const int32_t* sl = slots + o.slot;
  const double* sv = save + o.save;
  for (int k = threadIdx.x; k < o.r; k += blockDim.x) dc[k] = x[sl[k]] - sv[o.np + k];
  __syncthreads();
  for (int i = threadIdx.x; i < o.np; i += blockDim.x) {
    double s = sv[i];
    for (int k = 0; k < o.r; ++k) s += (double)o.Q[i + (size_t)k * o.np] * dc[k];
    x[sl[i]] = s;
  }
}

template <typename TF>
__global__ void __launch_bounds__(AT) k_scale_bwd(const ScaleOp<TF>* __restrict__ ops, const int32_t* __restrict__ slots,
                                                 double* __restrict__ x) {
  extern __shared__ double xs[];
  const ScaleOp<TF> o = ops[blockIdx.x];
  const int32_t* sl = slots + o.slot;
  for (int i = threadIdx.x; i < o.np; i += blockDim.x) xs[i] = x[sl[i]];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = warp; j < o.np; j += nw) {  // x_p <- U_p^{-1} x_p = Y^T x_p
    double v;
    trmv_lowerT_warp(o.Y, o.np, xs, j, v);
    if (lane == 0) x[sl[j]] = v;
  }
}

template <typename TF>
__global__ void __launch_bounds__(AT) k_elim_bwd(const ElimOp<TF>* __restrict__ ops, const int32_t* __restrict__ slots,
                                                double* __restrict__ x) {
  extern __shared__ double sh[];
  const ElimOp<TF> o = ops[blockIdx.x];
  const int32_t* sl = slots + o.slot;
  double* acc = sh;
  double* xn = sh + o.ns;
  for (int j = threadIdx.x; j < o.m; j += blockDim.x) xn[j] = x[sl[o.ns + j]];
  __syncthreads();
  const TF* XT = o.R + (size_t)o.ns * o.ns;
  for (int i = threadIdx.x; i < o.ns; i += blockDim.x) {  // acc = x_s - X_ns^T x_n
    double s = x[sl[i]];
    for (int j = 0; j < o.m; ++j) s -= (double)XT[i + (size_t)j * o.ns] * xn[j];
    acc[i] = s;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = warp; j < o.ns; j += nw) {  // x_s = U_s^{-1} acc
    double v;
    trmv_lowerT_warp(o.Y, o.ns, acc, j, v);
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

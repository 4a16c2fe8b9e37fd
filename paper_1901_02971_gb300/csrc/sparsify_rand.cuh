// Randomized compression of scaled interfaces: OrthS with the column-pivoted
// QR of A_pn replaced by a randomized range finder (Sec. 2.6.2 and Sec. 5
// name randomized low-rank methods as the alternative; method of Halko,
// Martinsson and Tropp, SIAM Review 2011, Algorithm 4.2, with a doubling
// sketch).  Per interface p of a colour, with A_pn = [A_pq1 ... A_pqk] (np x m,
// every current neighbour column) and ell_max = min(np, m):
//   1. ell = min(32, ell_max);
//   2. Y = A_pn Om[:, :ell], Om the m x ell_max Gaussian test matrix drawn
//      from its counter (Philox4x64-10 with Box-Muller, keyed by the seed,
//      the step and the cluster: entry (j, c) is a function of those alone, so
//      a larger sketch extends the smaller one);
//   3. the column-pivoted QR of Y orders an orthogonal basis Q of range(Y)
//      (the QR kernels run on Y as on a coupling block, without write-back);
//   4. W = Q^T A_pn (its first ell rows) and the squared trailing column
//      norms ||A_j||^2 - sum_{i<k} W_ij^2 (k = 0 .. ell; Q is orthogonal);
//   5. r = the first k whose largest trailing column norm is below
//      eps max_j ||A_j|| (the meaning of |R_kk| in a column-pivoted QR, the
//      truncation rule of Sec. 4); if there is none, or r > ell - 10, and
//      ell < ell_max, ell doubles and 2..5 run again; at ell_max with no such
//      k, r = ell;
//   6. as in Sec. 2.6.1: W_cn = W[:r] is written into p's block row and its
//      transposes into the neighbours' rows, A_cc = I, Q_pc = Q[:, :r], and
//      the size of p becomes r.
// The state of each interface (ell, its range, whether it is still active)
// lives in its task; the host only reads the active flags between rounds.
#pragma once

#include "cpqr_cluster.cuh"
#include "sketch.cuh"

namespace spand {

constexpr int RD_OVERSAMPLE = 10;  // sketch columns beyond the rank (HMT 2011, Sec. 4.2)
constexpr int RD_ELL0 = 32;        // first sketch width

template <typename T>
struct RandTask {
  T* Rp;                     // p's block row (leading dimension ldp)
  T* Om;                     // m_max x np sketch, column-major (leading dimension m_max)
  T* Y;                      // np x np capacity: Y = A_pn Om[:, :ell] (leading dimension np)
  T* W;                      // np x m_max capacity: W = Q^T A_pn, first ell rows (leading dimension np)
  T* Qc;                     // the basis formed from the QR of Y (np x np capacity, leading dimension np)
  int32_t* tcol;             // m_max: column of A_pn's column j in p's block row
  unsigned long long* res;   // np + 2: [k] max_j of the squared trailing norm at k (double bits); [np+1] max ||A_j||^2
  int32_t p, np, ldp, nbeg, nend, m_max;
  // device-side state
  int32_t m, ell, ell_prev, ell_max, active, rank;
};

__device__ __forceinline__ void rd_atomic_max(unsigned long long* a, double v) {
  atomicMax(a, (unsigned long long)__double_as_longlong(v));  // v >= 0: the bit order is the value order
}

// Setup of every task of a colour: the current width m (neighbour sizes
// after the earlier colours), the column map, max_j ||A_j||^2, ell.
// One CTA per task; the QR task of the sketch reads its width from vcur.
template <typename T>
__global__ void __launch_bounds__(256) k_rand_init(RandTask<T>* __restrict__ tasks, const CpqrNbr<T>* __restrict__ nbrs,
                                                   const int32_t* __restrict__ cur_size, int32_t* __restrict__ vcur) {
  RandTask<T>& d = tasks[blockIdx.x];
  __shared__ int cst[257];
  __shared__ double red[8];
  const int tid = threadIdx.x;
  const int nnb = d.nend - d.nbeg;
  if (nnb > 256) return;  // the host never builds such a task
  if (tid == 0) {
    int o = 0;
    for (int e = 0; e < nnb; ++e) {
      cst[e] = o;
      o += cur_size[nbrs[d.nbeg + e].q];
    }
    cst[nnb] = o;
  }
  __syncthreads();
  const int m = cst[nnb];
  for (int e = 0; e < nnb; ++e) {
    const CpqrNbr<T> nb = nbrs[d.nbeg + e];
    for (int jj = tid; jj < cst[e + 1] - cst[e]; jj += 256) d.tcol[cst[e] + jj] = nb.off_pq + jj;
  }
  __syncthreads();
  double mx = 0.0;  // max_j ||A_j||^2: a warp per column, lanes over rows (sums in T)
  for (int j = tid >> 5; j < m; j += 8) {
    const T* col = d.Rp + (size_t)d.tcol[j] * d.ldp;
    T s = T(0);
    for (int i = tid & 31; i < d.np; i += 32) s = fma(col[i], col[i], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    mx = fmax(mx, (double)s);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((tid & 31) == 0) red[tid >> 5] = mx;
  __syncthreads();
  for (int k = tid; k <= d.np + 1; k += 256) d.res[k] = 0ull;
  if (tid == 0) {
    double a = 0.0;
    for (int w = 0; w < 8; ++w) a = fmax(a, red[w]);
    d.res[d.np + 1] = (unsigned long long)__double_as_longlong(a);
    d.m = m;
    d.ell_max = min(d.np, m);
    d.ell = min(RD_ELL0, d.ell_max);
    d.ell_prev = 0;
    d.active = (m > 0 && d.np > 0) ? 1 : 0;
    d.rank = d.np;  // kept whole when there is nothing to compress against
    vcur[blockIdx.x] = d.ell;
  }
}

// Om[:, ell_prev:ell] of every active task (key (seed, step, cluster);
// FP64 sketches: entries as spand_sketch_gaussian draws them; FP32 sketches:
// the same Philox words, Box-Muller in FP32).
template <typename T>
__global__ void k_rand_omega(const RandTask<T>* __restrict__ tasks, uint64_t seed, int step) {
  const RandTask<T>& d = tasks[blockIdx.y];
  if (!d.active) return;
  const int m = d.m, nb = (m + 3) / 4, c0 = d.ell_prev, nc = d.ell - d.ell_prev;
  const uint64_t k1 = ((uint64_t)(uint32_t)step << 32) + (uint64_t)(uint32_t)d.p;
  const int total = nb * nc;  // <= (m_max / 4 + 1) * np
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const int j = c0 + t / nb, b = t - (t / nb) * nb;
    T* col = d.Om + (size_t)j * d.m_max;
    if constexpr (sizeof(T) == 4) {
      float z[4];
      philox_gauss4f(seed, k1, (uint64_t)j, (uint64_t)b, z);
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (4 * b + k < m) col[4 * b + k] = z[k];
    } else {
      double z[4];
      philox_gauss4(seed, k1, (uint64_t)j, (uint64_t)b, z);
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (4 * b + k < m) col[4 * b + k] = (T)z[k];
    }
  }
}

// Y[:, ell_prev:ell] = A_pn Om[:, ell_prev:ell], 32 x 32 tiles (tile
// blockIdx.x of task blockIdx.y), K = m in chunks of 32 staged in shared
// memory; thread (ty, tx) computes rows 4 ty .. 4 ty + 3 of column tx.
template <typename T>
__global__ void __launch_bounds__(256) k_rand_sketch(const RandTask<T>* __restrict__ tasks) {
  const RandTask<T>& d = tasks[blockIdx.y];
  if (!d.active) return;
  const int tr = (d.np + 31) / 32, tcn = (d.ell - d.ell_prev + 31) / 32;
  if ((int)blockIdx.x >= tr * tcn) return;
  const int r0 = 32 * ((int)blockIdx.x % tr), c0 = d.ell_prev + 32 * ((int)blockIdx.x / tr);
  __shared__ T a[32][33], b[32][33];
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  T acc[4] = {T(0), T(0), T(0), T(0)};
  for (int k0 = 0; k0 < d.m; k0 += 32) {
    for (int e = tid; e < 1024; e += 256) {
      // a[i][kk] = A(r0 + i, k0 + kk) and b[kk][c] = Om(k0 + kk, c0 + c), the
      // lanes of a warp along the rows of A and of Om (contiguous in both)
      const int i = e & 31, kk = e >> 5;
      const int k = k0 + kk;
      a[i][kk] = (r0 + i < d.np && k < d.m) ? d.Rp[(r0 + i) + (size_t)d.tcol[k] * d.ldp] : T(0);
      const int kb = k0 + i, c = kk;
      b[i][c] = (kb < d.m && c0 + c < d.ell) ? d.Om[kb + (size_t)(c0 + c) * d.m_max] : T(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      const T bv = b[kk][tx];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = fma(a[4 * ty + q][kk], bv, acc[q]);
    }
    __syncthreads();
  }
  const int c = c0 + tx;
  if (c < d.ell)
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (r0 + 4 * ty + q < d.np) d.Y[(r0 + 4 * ty + q) + (size_t)c * d.np] = acc[q];
}

// W[:ell, cols] = Q[:, :ell]^T A_pn[:, cols] for the 32 columns of block
// blockIdx.x, then the squared trailing norms t_j(k) = ||A_j||^2 -
// sum_{i<k} W_ij^2 (k = 0 .. ell), reduced to res[k] = max_j t_j(k).
// Thread (ty, tx): column tx, rows 4 ty .. 4 ty + 3 of each 32-row block.
template <typename T>
__global__ void __launch_bounds__(256) k_rand_project(RandTask<T>* __restrict__ tasks) {
  RandTask<T>& d = tasks[blockIdx.y];
  if (!d.active) return;
  const int j0 = 32 * (int)blockIdx.x;
  if (j0 >= d.m) return;
  __shared__ T q[32][33], a[32][33];
  __shared__ double wsq[32][33];
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  const int j = j0 + tx;
  const bool live = j < d.m;
  const T* colA = d.Rp + (size_t)(live ? d.tcol[j] : 0) * d.ldp;
  double nrm = 0.0;  // ||A_j||^2, summed by the warp of ty = 0 below
  double pre = 0.0;  // sum_{i<k} W_ij^2, carried by thread (0, tx)
  const int ell = d.ell;
  for (int i0 = 0; i0 < ell; i0 += 32) {
    T acc[4] = {T(0), T(0), T(0), T(0)};
    for (int k0 = 0; k0 < d.np; k0 += 32) {
      for (int e = tid; e < 1024; e += 256) {
        const int kk = e & 31, c = e >> 5;  // q[kk][c] = Q(k0 + kk, i0 + c); a[kk][c] = A(k0 + kk, j0 + c)
        const int k = k0 + kk;
        q[kk][c] = (k < d.np && i0 + c < ell) ? d.Qc[k + (size_t)(i0 + c) * d.np] : T(0);
        a[kk][c] = (k < d.np && j0 + c < d.m) ? d.Rp[k + (size_t)d.tcol[j0 + c] * d.ldp] : T(0);
      }
      __syncthreads();
      if (i0 == 0 && ty == 0)
        for (int kk = 0; kk < 32; ++kk) nrm += (double)a[kk][tx] * (double)a[kk][tx];
#pragma unroll 8
      for (int kk = 0; kk < 32; ++kk) {
        const T av = a[kk][tx];
#pragma unroll
        for (int s = 0; s < 4; ++s) acc[s] = fma(q[kk][4 * ty + s], av, acc[s]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int i = i0 + 4 * ty + s;
      if (live && i < ell) d.W[i + (size_t)j * d.np] = acc[s];
      wsq[4 * ty + s][tx] = (live && i < ell) ? (double)acc[s] * (double)acc[s] : 0.0;
    }
    __syncthreads();
    if (ty == 0)  // per column, t_j(k) for the block's rows k in order (wsq[k] becomes t_j(k))
      for (int ii = 0; ii < 32; ++ii) {
        const double w2 = wsq[ii][tx];
        wsq[ii][tx] = live ? fmax(nrm - pre, 0.0) : 0.0;
        pre += w2;  // rows at or beyond ell hold 0
      }
    __syncthreads();
    for (int ii = ty; ii < 32 && i0 + ii < ell; ii += 8) {  // max over the block's columns, a warp per row
      double t = wsq[ii][tx];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
      if (tx == 0) rd_atomic_max(&d.res[i0 + ii], t);
    }
    __syncthreads();
  }
  if (ty == 0) {  // k = ell
    double t = live ? fmax(nrm - pre, 0.0) : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
    if (tx == 0) rd_atomic_max(&d.res[ell], t);
  }
}

// The rank of every active task from res, and the next sketch width when
// the rank saturates the sketch (step 5); active[i] is read by the host.
template <typename T>
__global__ void k_rand_decide(RandTask<T>* __restrict__ tasks, int n, double eps, int32_t* __restrict__ vcur,
                              CpqrTask<T>* __restrict__ qtasks, int32_t* __restrict__ active) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  RandTask<T>& d = tasks[i];
  if (!d.active) {
    active[i] = 0;
    return;
  }
  const double a0sq = __longlong_as_double((long long)d.res[d.np + 1]);
  const double thr = eps * eps * a0sq;
  int r = -1;
  for (int k = 0; k <= d.ell; ++k)
    if (__longlong_as_double((long long)d.res[k]) < thr) {
      r = k;
      break;
    }
  if (d.ell == d.ell_max || (r >= 0 && r <= d.ell - RD_OVERSAMPLE)) {
    d.rank = r >= 0 ? r : d.ell;
    d.active = 0;
    qtasks[i].np = 0;  // the sketch's QR task has nothing left to do
    vcur[i] = 0;
  } else {
    d.ell_prev = d.ell;
    d.ell = min(2 * d.ell, d.ell_max);
    vcur[i] = d.ell;
    for (int k = 0; k <= d.ell; ++k) d.res[k] = 0ull;
  }
  active[i] = d.active;
}

// Step 6 for every task of the colour, grid (CTAs per task, tasks): W_cn
// into p's row and its transposes into the neighbours' rows, A_cc = I, the
// size of p (no other task of the colour reads it: the interfaces of one
// colour are not adjacent); a task with nothing to compress against keeps
// p whole with Q_pc = I.  The warps of a task's CTAs take columns, the
// lanes rows.
template <typename T>
__global__ void __launch_bounds__(256) k_rand_writeback(const RandTask<T>* __restrict__ tasks,
                                                        const CpqrNbr<T>* __restrict__ nbrs,
                                                        int32_t* __restrict__ cur_size) {
  const RandTask<T>& d = tasks[blockIdx.y];
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * 8 + (threadIdx.x >> 5), nw = gridDim.x * 8;
  const int np = d.np;
  const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
  if (d.m == 0 || np == 0) {
    for (int c = gw; c < np; c += nw)
      for (int i = lane; i < np; i += 32) d.Qc[i + (size_t)c * np] = (i == c) ? T(1) : T(0);
    if (lead) cur_size[d.p] = np;
    return;
  }
  const int r = d.rank;
  for (int j = gw; j < d.m; j += nw) {  // p's row
    T* dst = d.Rp + (size_t)d.tcol[j] * d.ldp;
    for (int i = lane; i < r; i += 32) dst[i] = d.W[i + (size_t)j * np];
  }
  int j = 0;  // transposes: columns of neighbour e are rows of its block A_qp
  for (int e = d.nbeg; e < d.nend; ++e) {
    const CpqrNbr<T> nb = nbrs[e];
    const int w = cur_size[nb.q];
    for (int i = gw; i < r; i += nw) {
      T* dst = nb.Rq + (size_t)(nb.off_qp + i) * nb.ldq;
      for (int jj = lane; jj < w; jj += 32) dst[jj] = d.W[i + (size_t)(j + jj) * np];
    }
    j += w;
  }
  for (int c = gw; c < r; c += nw)
    for (int i = lane; i < r; i += 32) d.Rp[i + (size_t)c * d.ldp] = (i == c) ? T(1) : T(0);
  if (lead) cur_size[d.p] = r;
}

}  // namespace spand

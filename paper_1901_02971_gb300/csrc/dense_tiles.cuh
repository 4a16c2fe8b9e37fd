// Dense tile building blocks shared by the factorization kernels.
//
// Storage convention: every dense matrix is column-major with a leading
// dimension; element (i, j) of a matrix at P with leading dimension ld is
// P[i + j*ld].  A cluster's block row [A_pp | A_pq1 | A_pq2 | ...] is one
// column-major |p| x W matrix (Sec. 2.2 block structure, one row per
// interface), so that Cholesky pivots, triangular solves, Schur updates and the
// column-pivoted QR of A_pn all read contiguous columns.
//
// Cholesky is taken in its upper form A = U^T U (U = L^T of Sec. 2.4), which
// keeps all reads along contiguous columns of the block row.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace spand {

constexpr int TB = 64;    // tile edge
constexpr int NT = 256;   // threads per CTA of the tile kernels
constexpr int KC = 16;    // k-chunk staged in shared memory

template <typename T>
struct TileSmem {
  T a[KC][TB + 1];
  T b[KC][TB + 1];
};

// acc[ii][jj] (row = tx + 16 ii, col = ty + 16 jj; tx = tid % 16, ty = tid / 16)
// += sum_{k < K} A[k + row*lda] * B[k + col*ldb]     ("TN": C += A^T B)
// Rows >= mi and columns >= nj read as zero.
template <typename T>
__device__ __forceinline__ void tn_acc(T (&acc)[4][4], const T* __restrict__ A, int lda, int mi,
                                       const T* __restrict__ B, int ldb, int nj, int K,
                                       TileSmem<T>& sm) {
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  for (int k0 = 0; k0 < K; k0 += KC) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = tid + NT * r;
      const int kk = e & (KC - 1);
      const int ii = e >> 4;
      const int k = k0 + kk;
      sm.a[kk][ii] = (k < K && ii < mi) ? A[k + (size_t)ii * lda] : T(0);
      sm.b[kk][ii] = (k < K && ii < nj) ? B[k + (size_t)ii * ldb] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
      T av[4], bv[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        av[q] = sm.a[kk][tx + 16 * q];
        bv[q] = sm.b[kk][ty + 16 * q];
      }
#pragma unroll
      for (int ii = 0; ii < 4; ++ii)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) acc[ii][jj] = fma(av[ii], bv[jj], acc[ii][jj]);
    }
    __syncthreads();
  }
}

template <typename T>
__device__ __forceinline__ void zero_acc(T (&acc)[4][4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
}

// C[row + col*ldc] -= acc for row < mi, col < nj.
template <typename T>
__device__ __forceinline__ void sub_store(const T (&acc)[4][4], T* C, int ldc, int mi, int nj) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int jj = 0; jj < 4; ++jj) {
    const int c = ty + 16 * jj;
    if (c >= nj) continue;
#pragma unroll
    for (int ii = 0; ii < 4; ++ii) {
      const int r = tx + 16 * ii;
      if (r < mi) C[r + (size_t)c * ldc] -= acc[ii][jj];
    }
  }
}

// Shared-memory square tile [TB][TB+1], s[i][j] = element (i, j).
template <typename T>
struct SqTile {
  T v[TB][TB + 1];
};

template <typename T>
__device__ __forceinline__ void load_tile(SqTile<T>& s, const T* P, int ld, int mi, int nj) {
  for (int e = threadIdx.x; e < TB * TB; e += NT) {
    const int i = e & (TB - 1), j = e >> 6;
    s.v[i][j] = (i < mi && j < nj) ? P[i + (size_t)j * ld] : T(0);
  }
}

template <typename T>
__device__ __forceinline__ void store_tile(const SqTile<T>& s, T* P, int ld, int mi, int nj) {
  for (int e = threadIdx.x; e < TB * TB; e += NT) {
    const int i = e & (TB - 1), j = e >> 6;
    if (i < mi && j < nj) P[i + (size_t)j * ld] = s.v[i][j];
  }
}

// In-place upper Cholesky of the nb x nb tile (upper triangle read/written).
// Returns false (for every thread) if a pivot is not positive.
template <typename T>
__device__ bool potrf_tile_upper(SqTile<T>& s, int nb) {
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int k = 0; k < nb; ++k) {
    if (threadIdx.x == 0) {
      const T d = s.v[k][k];
      if (!(d > T(0))) bad = 1;
      s.v[k][k] = sqrt(d > T(0) ? d : T(1));
    }
    __syncthreads();
    if (bad) return false;
    const T dk = s.v[k][k];
    for (int j = k + 1 + threadIdx.x; j < nb; j += NT) s.v[k][j] /= dk;
    __syncthreads();
    const int m = nb - k - 1;
    for (int e = threadIdx.x; e < m * m; e += NT) {
      const int i = k + 1 + e % m, j = k + 1 + e / m;
      if (i <= j) s.v[i][j] -= s.v[k][i] * s.v[k][j];
    }
    __syncthreads();
  }
  return true;
}

// B <- D B with D = U^{-T} the stored inverse of a diagonal tile (lower,
// zero above the diagonal), i.e. B <- U^{-T} B as one small GEMM instead of a
// serial substitution.  D, B in shared memory; each thread produces a 4x4
// patch; starts and ends synchronised.
template <typename T>
__device__ void apply_inv_tile(const SqTile<T>& D, SqTile<T>& B, int nb) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[4][4];
  zero_acc(acc);
  for (int l = 0; l < nb; ++l) {
    T dv[4], bv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      dv[q] = D.v[tx + 16 * q][l];
      bv[q] = B.v[l][ty + 16 * q];
    }
#pragma unroll
    for (int ii = 0; ii < 4; ++ii)
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) acc[ii][jj] = fma(dv[ii], bv[jj], acc[ii][jj]);
  }
  __syncthreads();
#pragma unroll
  for (int ii = 0; ii < 4; ++ii)
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) B.v[tx + 16 * ii][ty + 16 * jj] = acc[ii][jj];
  __syncthreads();
}

// In place: B <- U^{-T} B, U upper nb x nb, B nb x ncols (both in shared memory).
template <typename T>
__device__ void trsm_tile_upperT(const SqTile<T>& U, SqTile<T>& B, int nb, int ncols) {
  for (int i = 0; i < nb; ++i) {
    if (threadIdx.x < ncols) B.v[i][threadIdx.x] /= U.v[i][i];
    __syncthreads();
    const int m = nb - i - 1;
    for (int e = threadIdx.x; e < m * ncols; e += NT) {
      const int l = i + 1 + e / ncols, j = e % ncols;
      B.v[l][j] -= U.v[i][l] * B.v[i][j];
    }
    __syncthreads();
  }
}

}  // namespace spand

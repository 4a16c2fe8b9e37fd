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
struct TileSmem {  // two K chunks (double buffer)
  T a[2][KC][TB + 1];
  T b[2][KC][TB + 1];
};

// acc[ii][jj] (row = tx + 16 ii, col = ty + 16 jj; tx = tid % 16, ty = tid / 16)
// += sum_{k < K} A[k + row*lda] * B[k + col*ldb]     ("TN": C += A^T B)
// Rows >= mi and columns >= nj read as zero.
// UPPER: only the outputs on or above the diagonal of a diagonal tile are
// needed (rows tx + 16 ii > columns ty + 16 jj whenever ii > jj: those
// products are skipped and their accumulators stay zero).
template <typename T, bool UPPER = false>
__device__ __forceinline__ void tn_acc(T (&acc)[4][4], const T* __restrict__ A, int lda, int mi,
                                       const T* __restrict__ B, int ldb, int nj, int K,
                                       TileSmem<T>& sm) {
  // K in chunks of KC, double-buffered: chunk c + 1 is loaded into registers
  // while chunk c is multiplied from shared memory; one block barrier per chunk
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  T ra[4], rb[4];
  auto load = [&](int k0) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = tid + NT * r;
      const int kk = e & (KC - 1);
      const int ii = e >> 4;
      const int k = k0 + kk;
      ra[r] = (k < K && ii < mi) ? A[k + (size_t)ii * lda] : T(0);
      rb[r] = (k < K && ii < nj) ? B[k + (size_t)ii * ldb] : T(0);
    }
  };
  if (K <= 0) return;
  load(0);
  int buf = 0;
  for (int k0 = 0; k0 < K; k0 += KC) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = tid + NT * r;
      sm.a[buf][e & (KC - 1)][e >> 4] = ra[r];
      sm.b[buf][e & (KC - 1)][e >> 4] = rb[r];
    }
    __syncthreads();
    if (k0 + KC < K) load(k0 + KC);
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
      T av[4], bv[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        av[q] = sm.a[buf][kk][tx + 16 * q];
        bv[q] = sm.b[buf][kk][ty + 16 * q];
      }
#pragma unroll
      for (int ii = 0; ii < 4; ++ii)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj)
          if (!UPPER || ii <= jj) acc[ii][jj] = fma(av[ii], bv[jj], acc[ii][jj]);
    }
    buf ^= 1;
  }
  __syncthreads();  // the caller may reuse the buffers
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

// Upper Cholesky of the nb x nb diagonal tile s (A = U^T U, upper triangle
// read and overwritten with U, lower triangle left as loaded) fused with the
// inverse D = U^{-T} (lower, TB x TB, identity beyond nb).  Right-looking,
// two pivot rows per step: rows k and k + 1 of A and of D are published to
// shared memory, every thread forms the 2 x 2 pivot block from them,
//   U_kk = sqrt(A_kk), U_k. = A_k. / U_kk,
//   U_{k+1,k+1} = sqrt(A_{k+1,k+1} - U_{k,k+1}^2),
//   U_{k+1,.} = (A_{k+1,.} - U_{k,k+1} U_k.) / U_{k+1,k+1},
//   D_k. <- D_k. / U_kk,  D_{k+1,.} <- (D_{k+1,.} - U_{k,k+1} D_k.) / U_{k+1,k+1},
// and updates the 4 x 4 elements it holds in registers (rows tx + 16a,
// columns ty + 16b) with the rank-2 terms:
//   A_ij -= U_ki U_kj + U_{k+1,i} U_{k+1,j} (k + 1 < i <= j),
//   D_i. -= U_ki D_k. + U_{k+1,i} D_{k+1,.} (i > k + 1)   (row ops of L^{-1}, L = U^T).
// One block barrier per pair of rows (the row buffers alternate); 1 / U_kk
// comes from one reciprocal square root.  Returns false (for every thread) if
// a pivot is not positive; nothing is stored then.
template <typename T>
__device__ bool potrf_inv_tile(SqTile<T>& s, SqTile<T>& D, int nb) {
  __shared__ T rowA[2][2][TB], rowD[2][2][TB];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T a[4][4], d[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = tx + 16 * p, j = ty + 16 * q;
      a[p][q] = s.v[i][j];
      d[p][q] = (i == j) ? T(1) : T(0);
    }
  for (int k = 0; k < nb; k += 2) {
    const int par = (k >> 1) & 1;
    const bool two = k + 1 < nb;
    const int k1 = two ? k + 1 : k;  // a single last row repeats row k (unused)
#pragma unroll
    for (int p = 0; p < 4; ++p) {  // owners of rows k, k + 1 publish them (compile-time register indices)
      const int i = tx + 16 * p;
      if (i == k || i == k1) {
        const int w = i == k ? 0 : 1;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          rowA[par][w][ty + 16 * q] = a[p][q];
          rowD[par][w][ty + 16 * q] = d[p][q];
        }
      }
    }
    __syncthreads();
    const T a00 = rowA[par][0][k];
    if (!(a00 > T(0))) return false;  // uniform: every thread read the same pivot
    const T r0 = rsqrt(a00), u00 = a00 * r0;
    const T u01 = two ? rowA[par][0][k1] * r0 : T(0);
    const T s11 = two ? rowA[par][1][k1] - u01 * u01 : T(1);
    if (!(s11 > T(0))) return false;
    const T r1 = rsqrt(s11), u11 = s11 * r1;
    T u0i[4], u1i[4], u0j[4], u1j[4], d0[4], d1[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int ci = tx + 16 * q, cj = ty + 16 * q;
      u0i[q] = rowA[par][0][ci] * r0;
      u0j[q] = rowA[par][0][cj] * r0;
      d0[q] = rowD[par][0][cj] * r0;
      u1i[q] = two ? (rowA[par][1][ci] - u01 * u0i[q]) * r1 : T(0);
      u1j[q] = two ? (rowA[par][1][cj] - u01 * u0j[q]) * r1 : T(0);
      d1[q] = two ? (rowD[par][1][cj] - u01 * d0[q]) * r1 : T(0);
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int i = tx + 16 * p;
      if (i == k) {  // finalise row k of U and of D
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = ty + 16 * q;
          if (j == k) a[p][q] = u00;
          else if (j > k) a[p][q] = u0j[q];
          d[p][q] = d0[q];
        }
      } else if (two && i == k1) {  // finalise row k + 1
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = ty + 16 * q;
          if (j == k1) a[p][q] = u11;
          else if (j > k1) a[p][q] = u1j[q];
          d[p][q] = d1[q];
        }
      } else if (i > k1) {
        // U's upper triangle: column block q >= row block p; D's lower
        // triangle: q <= p (the other blocks are zero in D and unused in U)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = ty + 16 * q;
          if (q >= p && j >= i) a[p][q] = fma(-u1i[p], u1j[q], fma(-u0i[p], u0j[q], a[p][q]));
          if (q <= p) d[p][q] = fma(-u1i[p], d1[q], fma(-u0i[p], d0[q], d[p][q]));
        }
      }
    }
  }
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = tx + 16 * p, j = ty + 16 * q;
      if (i <= j) s.v[i][j] = a[p][q];
      D.v[i][j] = d[p][q];
    }
  __syncthreads();
  return true;
}

// B <- D B with D = U^{-T} the stored inverse of a diagonal tile (lower,
// zero above the diagonal), i.e. B <- U^{-T} B as one small GEMM instead of a
// serial substitution.  D, B in shared memory; each thread produces a 4x4
// patch; starts and ends synchronised.
// D is lower triangular: for l in the 16-row block lb, the rows tx + 16 ii
// with ii < lb lie above l, where D is zero, so their products are skipped
// (uniformly over the CTA).
template <typename T>
__device__ void apply_inv_tile(const SqTile<T>& D, SqTile<T>& B, int nb) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[4][4];
  zero_acc(acc);
#pragma unroll
  for (int lb = 0; lb < 4; ++lb) {
    const int le = min(nb, 16 * lb + 16);
    for (int l = 16 * lb; l < le; ++l) {
      T dv[4], bv[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        dv[q] = D.v[tx + 16 * q][l];
        bv[q] = B.v[l][ty + 16 * q];
      }
#pragma unroll
      for (int ii = lb; ii < 4; ++ii)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) acc[ii][jj] = fma(dv[ii], bv[jj], acc[ii][jj]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int ii = 0; ii < 4; ++ii)
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) B.v[tx + 16 * ii][ty + 16 * jj] = acc[ii][jj];
  __syncthreads();
}

}  // namespace spand

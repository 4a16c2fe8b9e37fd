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

constexpr int TB = 64;    // tile edge of the factorization kernels
constexpr int NT = 256;   // threads per CTA of the tile kernels (64-row tiles)
constexpr int KC = 16;    // k-chunk staged in shared memory
constexpr int TB2 = 32;   // tile edge of the FP64 pivot Cholesky (shorter dependent chains)

// Tiles of edge B are processed by PR x PC threads, each holding a 4 x CB
// patch: rows tx + PR ii (ii < 4), columns ty + PC jj (jj < CB),
// tx = tid % PR, ty = tid / PR.  64-tiles: 16 x 16 threads with 4 x 4
// patches.  32-tiles (the FP64 pivot Cholesky): 8 x 16 threads with 4 x 2
// patches -- four warps, one per SM sub-partition, because a warp-wide FP64
// FMA occupies a sub-partition's FP64 unit for tens of cycles on this GPU,
// so a tile held by two warps leaves half of the SM's FP64 units idle.
template <int B>
struct TileGeom {
  static constexpr int PR = B / 4;                  // threads along the rows
  static constexpr int PC = B == 32 ? 16 : B / 4;   // threads along the columns
  static constexpr int CB = B / PC;                 // columns per thread
  static constexpr int NTH = PR * PC;               // threads per CTA
  // row block ii lies entirely below column block jj (no element with row <= column)
  __host__ __device__ static constexpr bool below(int ii, int jj) { return ii * PR >= PC * (jj + 1); }
  // row block ii lies entirely above column block jj (no element with row >= column)
  __host__ __device__ static constexpr bool above(int ii, int jj) { return (ii + 1) * PR <= jj * PC; }
};

template <typename T, int B = TB>
struct TileSmemB {  // two K chunks (double buffer)
  T a[2][KC][B + 1];
  T b[2][KC][B + 1];
};
template <typename T>
using TileSmem = TileSmemB<T, TB>;

// acc[ii][jj] (row = tx + PR ii, col = ty + PC jj)
// += sum_{k < K} A[k + row*lda] * B[k + col*ldb]     ("TN": C += A^T B)
// Rows >= mi and columns >= nj read as zero.
// UPPER: only the outputs on or above the diagonal of a diagonal tile are
// needed (the patches whose row block lies entirely below their column
// block are skipped and their accumulators stay zero).
template <typename T, bool UPPER = false, int B = TB>
__device__ __forceinline__ void tn_acc(T (&acc)[4][TileGeom<B>::CB], const T* __restrict__ A, int lda, int mi,
                                       const T* __restrict__ Bm, int ldb, int nj, int K,
                                       TileSmemB<T, B>& sm) {
  // K in chunks of KC, double-buffered: chunk c + 1 is loaded into registers
  // while chunk c is multiplied from shared memory; one block barrier per chunk
  using G = TileGeom<B>;
  constexpr int PR = G::PR, PC = G::PC, CB = G::CB, NTH = G::NTH;
  constexpr int NL = KC * B / NTH;  // elements of each operand loaded per thread per chunk
  const int tid = threadIdx.x;
  const int tx = tid % PR, ty = tid / PR;
  T ra[NL], rb[NL];
  auto load = [&](int k0) {
#pragma unroll
    for (int r = 0; r < NL; ++r) {
      const int e = tid + NTH * r;
      const int kk = e & (KC - 1);
      const int ii = e >> 4;
      const int k = k0 + kk;
      ra[r] = (k < K && ii < mi) ? A[k + (size_t)ii * lda] : T(0);
      rb[r] = (k < K && ii < nj) ? Bm[k + (size_t)ii * ldb] : T(0);
    }
  };
  if (K <= 0) return;
  load(0);
  int buf = 0;
  for (int k0 = 0; k0 < K; k0 += KC) {
#pragma unroll
    for (int r = 0; r < NL; ++r) {
      const int e = tid + NTH * r;
      sm.a[buf][e & (KC - 1)][e >> 4] = ra[r];
      sm.b[buf][e & (KC - 1)][e >> 4] = rb[r];
    }
    __syncthreads();
    if (k0 + KC < K) load(k0 + KC);
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
      T av[4], bv[CB];
#pragma unroll
      for (int q = 0; q < 4; ++q) av[q] = sm.a[buf][kk][tx + PR * q];
#pragma unroll
      for (int q = 0; q < CB; ++q) bv[q] = sm.b[buf][kk][ty + PC * q];
#pragma unroll
      for (int ii = 0; ii < 4; ++ii)
#pragma unroll
        for (int jj = 0; jj < CB; ++jj)
          if (!UPPER || !G::below(ii, jj)) acc[ii][jj] = fma(av[ii], bv[jj], acc[ii][jj]);
    }
    buf ^= 1;
  }
  __syncthreads();  // the caller may reuse the buffers
}

template <typename T, int CB>
__device__ __forceinline__ void zero_acc(T (&acc)[4][CB]) {
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < CB; ++j) acc[i][j] = T(0);
}

// C[row + col*ldc] -= acc for row < mi, col < nj.
template <int B = TB, typename T>
__device__ __forceinline__ void sub_store(const T (&acc)[4][TileGeom<B>::CB], T* C, int ldc, int mi, int nj) {
  using G = TileGeom<B>;
  const int tx = threadIdx.x % G::PR, ty = threadIdx.x / G::PR;
#pragma unroll
  for (int jj = 0; jj < G::CB; ++jj) {
    const int c = ty + G::PC * jj;
    if (c >= nj) continue;
#pragma unroll
    for (int ii = 0; ii < 4; ++ii) {
      const int r = tx + G::PR * ii;
      if (r < mi) C[r + (size_t)c * ldc] -= acc[ii][jj];
    }
  }
}

// Shared-memory square tile [B][B+1], s[i][j] = element (i, j).
template <typename T, int B = TB>
struct SqTileB {
  static constexpr int E = B;
  T v[B][B + 1];
};
template <typename T>
using SqTile = SqTileB<T, TB>;

template <typename T, int B>
__device__ __forceinline__ void load_tile(SqTileB<T, B>& s, const T* P, int ld, int mi, int nj) {
  for (int e = threadIdx.x; e < B * B; e += TileGeom<B>::NTH) {
    const int i = e % B, j = e / B;
    s.v[i][j] = (i < mi && j < nj) ? P[i + (size_t)j * ld] : T(0);
  }
}

// The same load issued as asynchronous copies (cp.async, one element each,
// zero-filled outside mi x nj); complete with cp_async_wait_all() and a block
// barrier before reading the tile.
template <typename T, int B>
__device__ __forceinline__ void load_tile_async(SqTileB<T, B>& s, const T* P, int ld, int mi, int nj) {
  for (int e = threadIdx.x; e < B * B; e += TileGeom<B>::NTH) {
    const int i = e % B, j = e / B;
    const bool in = i < mi && j < nj;
    const T* src = in ? P + i + (size_t)j * ld : P;
    const unsigned dst = (unsigned)__cvta_generic_to_shared(&s.v[i][j]);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(dst), "l"(src), "n"(sizeof(T)),
                 "r"(in ? (int)sizeof(T) : 0)
                 : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

template <typename T, int B>
__device__ __forceinline__ void store_tile(const SqTileB<T, B>& s, T* P, int ld, int mi, int nj) {
  for (int e = threadIdx.x; e < B * B; e += TileGeom<B>::NTH) {
    const int i = e % B, j = e / B;
    if (i < mi && j < nj) P[i + (size_t)j * ld] = s.v[i][j];
  }
}

// Upper Cholesky of the nb x nb diagonal tile s (A = U^T U, upper triangle
// read and overwritten with U, lower triangle left as loaded) fused with the
// inverse D = U^{-T} (lower, B x B, identity beyond nb).  Right-looking,
// two pivot rows per step.  The owners of rows k and k + 1 of A and of D
// publish them to shared memory; after a block barrier warp 0 alone forms
// the 2 x 2 pivot block and the scaled rows (lane l takes the columns
// l, l + 32, ...),
//   U_kk = sqrt(A_kk), U_k. = A_k. / U_kk,
//   U_{k+1,k+1} = sqrt(A_{k+1,k+1} - U_{k,k+1}^2),
//   U_{k+1,.} = (A_{k+1,.} - U_{k,k+1} U_k.) / U_{k+1,k+1},
//   D_k. <- D_k. / U_kk,  D_{k+1,.} <- (D_{k+1,.} - U_{k,k+1} D_k.) / U_{k+1,k+1},
// and publishes them; after a second barrier every thread updates the
// 4 x CB elements it holds in registers (rows tx + PR a, columns ty + PC b)
// with the rank-2 terms:
//   A_ij -= U_ki U_kj + U_{k+1,i} U_{k+1,j} (k + 1 < i <= j),
//   D_i. -= U_ki D_k. + U_{k+1,i} D_{k+1,.} (i > k + 1)   (row ops of L^{-1}, L = U^T).
// The pivot scalars and the row scalings are FP64 work that every warp
// would otherwise repeat on its own sub-partition (on this GPU a warp-wide
// FP64 instruction occupies a sub-partition for tens of cycles), so one warp
// does them once: fewer FP64 instructions per step on the critical path and
// in total.  The row and result buffers alternate with the step parity.
// 1 / U_kk comes from one reciprocal square root.  Returns false (for every
// thread) if a pivot is not positive; nothing is stored then.
template <typename T, int B>
__device__ bool potrf_inv_tile(SqTileB<T, B>& s, SqTileB<T, B>& D, int nb) {
  using G = TileGeom<B>;
  constexpr int PR = G::PR, PC = G::PC, CB = G::CB;
  __shared__ T rowA[2][2][B], rowD[2][2][B];        // raw rows k, k + 1
  __shared__ T scU[2][2][B], scD[2][2][B];          // scaled rows of U and of D
  __shared__ T scP[2][2];                           // U_kk, U_{k+1,k+1}
  __shared__ int okP[2];
  const int tx = threadIdx.x % PR, ty = threadIdx.x / PR;
  T a[4][CB], d[4][CB];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < CB; ++q) {
      const int i = tx + PR * p, j = ty + PC * q;
      a[p][q] = s.v[i][j];
      d[p][q] = (i == j) ? T(1) : T(0);
    }
  for (int k = 0; k < nb; k += 2) {
    const int par = (k >> 1) & 1;
    const bool two = k + 1 < nb;
    const int k1 = two ? k + 1 : k;  // a single last row repeats row k (unused)
#pragma unroll
    for (int p = 0; p < 4; ++p) {  // owners of rows k, k + 1 publish them (compile-time register indices)
      const int i = tx + PR * p;
      if (i == k || i == k1) {
        const int w = i == k ? 0 : 1;
#pragma unroll
        for (int q = 0; q < CB; ++q) {
          rowA[par][w][ty + PC * q] = a[p][q];
          rowD[par][w][ty + PC * q] = d[p][q];
        }
      }
    }
    __syncthreads();
    if (threadIdx.x < 32) {  // warp 0: the pivot block and the scaled rows
      const T a00 = rowA[par][0][k];
      const T r0 = rsqrt(a00), u00 = a00 * r0;
      const T u01 = two ? rowA[par][0][k1] * r0 : T(0);
      const T s11 = two ? rowA[par][1][k1] - u01 * u01 : T(1);
      const T r1 = rsqrt(s11), u11 = s11 * r1;
      for (int j = threadIdx.x; j < B; j += 32) {
        const T v0 = rowA[par][0][j] * r0, e0 = rowD[par][0][j] * r0;
        scU[par][0][j] = v0;
        scD[par][0][j] = e0;
        scU[par][1][j] = two ? (rowA[par][1][j] - u01 * v0) * r1 : T(0);
        scD[par][1][j] = two ? (rowD[par][1][j] - u01 * e0) * r1 : T(0);
      }
      if (threadIdx.x == 0) {
        scP[par][0] = u00;
        scP[par][1] = u11;
        okP[par] = (a00 > T(0)) && (s11 > T(0));
      }
    }
    __syncthreads();
    if (!okP[par]) return false;  // uniform: every thread reads the same flag
    T u0i[4], u1i[4], u0j[CB], u1j[CB], d0[CB], d1[CB];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int ci = tx + PR * q;
      u0i[q] = scU[par][0][ci];
      u1i[q] = scU[par][1][ci];
    }
#pragma unroll
    for (int q = 0; q < CB; ++q) {
      const int cj = ty + PC * q;
      u0j[q] = scU[par][0][cj];
      u1j[q] = scU[par][1][cj];
      d0[q] = scD[par][0][cj];
      d1[q] = scD[par][1][cj];
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int i = tx + PR * p;
      if (i == k) {  // finalise row k of U and of D
#pragma unroll
        for (int q = 0; q < CB; ++q) {
          const int j = ty + PC * q;
          if (j == k) a[p][q] = scP[par][0];
          else if (j > k) a[p][q] = u0j[q];
          d[p][q] = d0[q];
        }
      } else if (two && i == k1) {  // finalise row k + 1
#pragma unroll
        for (int q = 0; q < CB; ++q) {
          const int j = ty + PC * q;
          if (j == k1) a[p][q] = scP[par][1];
          else if (j > k1) a[p][q] = u1j[q];
          d[p][q] = d1[q];
        }
      } else if (i > k1) {
        // U's upper triangle and D's lower triangle: patches entirely on the
        // other side of the diagonal are skipped (they are zero in D and
        // unused in U); D's entries above the diagonal stay zero because
        // rows k, k + 1 of D are zero there
#pragma unroll
        for (int q = 0; q < CB; ++q) {
          const int j = ty + PC * q;
          if (!G::below(p, q) && j >= i) a[p][q] = fma(-u1i[p], u1j[q], fma(-u0i[p], u0j[q], a[p][q]));
          if (!G::above(p, q)) d[p][q] = fma(-u1i[p], d1[q], fma(-u0i[p], d0[q], d[p][q]));
        }
      }
    }
  }
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < CB; ++q) {
      const int i = tx + PR * p, j = ty + PC * q;
      if (i <= j) s.v[i][j] = a[p][q];
      D.v[i][j] = d[p][q];
    }
  __syncthreads();
  return true;
}

// B <- D B with D = U^{-T} the stored inverse of a diagonal tile (lower,
// zero above the diagonal), i.e. B <- U^{-T} B as one small GEMM instead of a
// serial substitution.  D, B in shared memory; each thread produces a 4x4
// patch; starts and ends synchronised.  For l in the PR-row block lb, the
// rows tx + PR ii with ii < lb lie above l, where D is zero, so their
// products are skipped (uniformly over the CTA).
template <typename T, int B>
__device__ void apply_inv_tile(const SqTileB<T, B>& D, SqTileB<T, B>& Bt, int nb) {
  using G = TileGeom<B>;
  constexpr int PR = G::PR, PC = G::PC, CB = G::CB;
  const int tx = threadIdx.x % PR, ty = threadIdx.x / PR;
  T acc[4][CB];
  zero_acc(acc);
#pragma unroll
  for (int lb = 0; lb < 4; ++lb) {
    const int le = min(nb, PR * lb + PR);
    for (int l = PR * lb; l < le; ++l) {
      T dv[4], bv[CB];
#pragma unroll
      for (int q = 0; q < 4; ++q) dv[q] = D.v[tx + PR * q][l];
#pragma unroll
      for (int q = 0; q < CB; ++q) bv[q] = Bt.v[l][ty + PC * q];
#pragma unroll
      for (int ii = lb; ii < 4; ++ii)
#pragma unroll
        for (int jj = 0; jj < CB; ++jj) acc[ii][jj] = fma(dv[ii], bv[jj], acc[ii][jj]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int ii = 0; ii < 4; ++ii)
#pragma unroll
    for (int jj = 0; jj < CB; ++jj) Bt.v[tx + PR * ii][ty + PC * jj] = acc[ii][jj];
  __syncthreads();
}

}  // namespace spand

// Two-sided transform of the coupling blocks for the simultaneous
// sparsification order: every interface p of a level takes its column-pivoted
// QR from the same scaled matrix (no W_cn write-back), and afterwards every
// coupling block becomes
//     A_pq <- Q_pc^T A_pq Q_qc      (r_p x r_q, Sec. 2.6.1 applied from both
//                                    sides at once),
// written into the top-left corner of A_pq in p's block row and, transposed,
// of A_qp in q's row.  The kept matrix is the c-c principal submatrix of the
// orthogonal similarity diag(Q_p)^T A diag(Q_p), so it stays SPD.
//
// Two launches of one batched GEMM kernel: Y = A_pq Q_qc (all edges), then
// X = Q_pc^T Y (all edges).  Every read of A_pq happens in the first launch,
// every write in the second, so the in-place update is race-free.  Extents
// that are ranks are read on the device from the rank array (the host plans
// the grid with the sizes as upper bounds); tiles beyond a rank return.
#pragma once

#include <cstdint>

namespace spand {

template <typename T>
struct SimGemm {      // C (M x N) = op(A) (M x K) B (K x N); column-major
  const T* A;         // transA = 0: A[i + k*lda]; transA = 1: A[k + i*lda]
  const T* B;         // B[k + j*ldb]
  T* C;               // C[i + j*ldc]
  T* C2;              // if not null: C2[j + i*ldc2] = C(i, j) (the transposed copy)
  int32_t lda, ldb, ldc, ldc2;
  int32_t m, n, k;    // extents; m and n are upper bounds when mi / ni >= 0
  int32_t mi, ni;     // M = min(m, ranks[mi]) if mi >= 0, N likewise
  int32_t transA;
  int32_t tiles_m;    // ceil(m / SG_TM): the tiles of one descriptor are tiles_m x ceil(n / SG_TN)
};

constexpr int SG_TM = 64, SG_TN = 32, SG_TK = 32, SG_NT = 256;

// One CTA per 64 x 32 output tile of one descriptor; toff[d] = first tile of
// descriptor d (prefix sums, toff[nd] = grid size).  Each warp owns 8 rows
// of the tile and each lane one column.
template <typename T>
__global__ void __launch_bounds__(SG_NT) k_sim_gemm(const SimGemm<T>* __restrict__ g,
                                                    const int32_t* __restrict__ toff, int nd,
                                                    const int32_t* __restrict__ ranks) {
  const int bid = blockIdx.x;
  int lo = 0, hi = nd - 1;  // last d with toff[d] <= bid
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (toff[mid] <= bid) lo = mid;
    else hi = mid - 1;
  }
  const SimGemm<T> G = g[lo];
  const int M = G.mi >= 0 ? min(G.m, ranks[G.mi]) : G.m;
  const int N = G.ni >= 0 ? min(G.n, ranks[G.ni]) : G.n;
  const int K = G.k;
  const int local = bid - toff[lo];
  const int i0 = (local % G.tiles_m) * SG_TM, j0 = (local / G.tiles_m) * SG_TN;
  if (i0 >= M || j0 >= N) return;  // also a negative (error) rank
  __shared__ T As[SG_TK][SG_TM + 1];
  __shared__ T Bs[SG_TK][SG_TN + 1];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  T acc[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) acc[r] = T(0);
  for (int k0 = 0; k0 < K; k0 += SG_TK) {
    for (int e = tid; e < SG_TM * SG_TK; e += SG_NT) {
      int ii, kk;
      if (G.transA) { kk = e % SG_TK; ii = e / SG_TK; }
      else { ii = e % SG_TM; kk = e / SG_TM; }
      const int gi = i0 + ii, gk = k0 + kk;
      T v = T(0);
      if (gi < M && gk < K) v = G.transA ? G.A[(size_t)gi * G.lda + gk] : G.A[(size_t)gk * G.lda + gi];
      As[kk][ii] = v;
    }
    for (int e = tid; e < SG_TK * SG_TN; e += SG_NT) {
      const int kk = e % SG_TK, jj = e / SG_TK;
      const int gk = k0 + kk, gj = j0 + jj;
      Bs[kk][jj] = (gk < K && gj < N) ? G.B[(size_t)gj * G.ldb + gk] : T(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < SG_TK; ++kk) {
      const T b = Bs[kk][lane];
#pragma unroll
      for (int r = 0; r < 8; ++r) acc[r] += As[kk][w * 8 + r] * b;
    }
    __syncthreads();
  }
  const int j = j0 + lane;
  if (j >= N) return;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int i = i0 + w * 8 + r;
    if (i < M) {
      G.C[(size_t)j * G.ldc + i] = acc[r];
      if (G.C2) G.C2[(size_t)i * G.ldc2 + j] = acc[r];
    }
  }
}

}  // namespace spand

// Batched kernels of the level-by-level spaND factorization (Algorithm 2).
// Every kernel processes all clusters of one step (or one colour) in a single
// launch; descriptors are built by the host scheduler once the step's block
// sizes are known.
#pragma once

#include "dense_tiles.cuh"

namespace spand {

// ---------------------------------------------------------------- descriptors

// Tile bandwidth of a pivot block: U's tile (I, J), I <= J, can be nonzero
// only if J - I <= bw (0 = dense).  A Cholesky factor keeps the envelope of
// its matrix (no fill above the first nonzero of a column), so for a pivot
// block that is still a piece of the sparse A (a leaf interior, eliminated
// first, with its vertices in lexicographic order: a band of one grid layer)
// the tiles outside the band hold exact zeros before and after the
// factorization, and the kernels skip them: same result, far fewer flops.
template <typename T>
struct RowDesc {      // a cluster's block row or its diagonal block
  T* R;               // column-major, leading dimension ld
  int32_t n;          // rows (cluster size)
  int32_t ld;
  T* dinv;            // ceil(n/64) tiles of 64x64: inverses U_kk^{-T} of the diagonal tiles
  int32_t bw;         // tile bandwidth of U in 64-tiles (0 = dense)
  int32_t bw2;        // the same in 32-tiles (FP64 pivot factorization)
  int32_t band;       // element half-bandwidth of the block (0 = dense or not known)
  int32_t pad;
};

template <typename T>
struct TrsmTask {     // B <- U^{-T} B: U upper n x n, B n x nc (rows < i_start of B are zero)
  const T* U;
  const T* dinv;      // inverses of U's diagonal 64x64 tiles (see RowDesc)
  T* B;
  int32_t n, ldu, ldb, nc, i_start, bw;  // bw: tile bandwidth of U (0 = dense)
};

template <typename T>
struct SchurBlock {   // target block (a, b), a <= b, of the elimination update (Sec. 2.4)
  T* C1;              // block (a, b) in a's row: rows |a|, cols |b|
  T* C2;              // block (b, a) in b's row (nullptr when a == b)
  int32_t ld1, ld2, rows, cols;
  int32_t cbeg, cend; // contributors
};

template <typename T>
struct SchurContrib { // one eliminated separator s adjacent to both a and b
  const T* Xa;        // X^T columns of a inside s's row: Xa[k + i*lds], k < ns
  const T* Xb;
  int32_t lds, ns;
  int32_t owner, pad; // s (index in the step's cluster list; host bookkeeping)
};

struct SchurTile {
  int32_t block, i0, j0;
};

template <typename T>
struct CopyTask {     // dst[r + c*ldd] = src[r + c*lds] (trans = 0) or src[c + r*lds] (trans = 1)
  const T* src;
  T* dst;
  int32_t lds, ldd, rows, cols, trans, pad;
};


// Programmatic dependent launch: the tile Cholesky's phases (and the banded
// Cholesky) are launched so that a kernel's CTAs may be scheduled while the
// previous kernel drains.
// Every CTA first waits for the previous grid's completion (and visibility of
// its writes) -- also the CTAs that then find no work, so that a grid never
// completes before its predecessor -- and signals the next grid once its own
// stores are issued.  Without the launch attribute both are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ---------------------------------------------------------------- assembly

// Scatter A's values into the step-1 block rows: rows[dst_row[e]][dst_off[e]] = vals[e].
template <typename T>
__global__ void k_assemble(const double* __restrict__ vals, const int32_t* __restrict__ dst_row,
                           const int64_t* __restrict__ dst_off, T* const* __restrict__ rows, int64_t nnz) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = dst_row[e];
    if (r >= 0) rows[r][dst_off[e]] = (T)vals[e];
  }
}

// ---------------------------------------------------------------- tiled Cholesky

// Tiled upper Cholesky of a batch of pivot blocks, B x B tiles (B = 64, or
// 32 for the FP64 pivots, whose per-SM rate makes the dependent chain of
// diagonal-tile factor -> tile solve -> trailing tile update the cost: a
// smaller tile shortens every link of that chain).  dinv holds ceil(n/B)
// tiles of B x B (the inverses U_kk^{-T} of phase 1); bw counts B-tiles.

// Tile step k, phase 1: factor diagonal tile (k, k) of every block and store
// the inverse of its factor, U_kk^{-T}, for the tile solves of phase 2.
template <typename T, int B = TB>
__global__ void __launch_bounds__(TileGeom<B>::NTH) k_potrf_diag(const RowDesc<T>* __restrict__ rows, int k,
                                                                 int* info) {
  extern __shared__ __align__(16) unsigned char smraw[];
  SqTileB<T, B>& s = *reinterpret_cast<SqTileB<T, B>*>(smraw);
  SqTileB<T, B>& Id = *reinterpret_cast<SqTileB<T, B>*>(smraw + sizeof(SqTileB<T, B>));
  pdl_wait();
  const RowDesc<T> d = rows[blockIdx.x];
  const int k0 = k * B;
  if (k0 >= d.n) return;
  const int nb = min(B, d.n - k0);
  T* P = d.R + k0 + (size_t)k0 * d.ld;
  load_tile(s, P, d.ld, nb, nb);
  __syncthreads();
  if (!potrf_inv_tile(s, Id, nb)) {
    if (threadIdx.x == 0) atomicCAS(info, 0, (int)blockIdx.x + 1);
    return;
  }
  store_tile(s, P, d.ld, nb, nb);
  store_tile(Id, d.dinv + (size_t)k * B * B, B, B, B);
  pdl_trigger();
}

// Tile step k, phase 2: U_kj = U_kk^{-T} A_kj for the tiles j > k of the diagonal block.
template <typename T, int B = TB>
__global__ void __launch_bounds__(TileGeom<B>::NTH) k_potrf_trsm(const RowDesc<T>* __restrict__ rows, int k) {
  extern __shared__ __align__(16) unsigned char smraw[];
  SqTileB<T, B>& D = *reinterpret_cast<SqTileB<T, B>*>(smraw);
  SqTileB<T, B>& Bt = *reinterpret_cast<SqTileB<T, B>*>(smraw + sizeof(SqTileB<T, B>));
  pdl_wait();
  const RowDesc<T> d = rows[blockIdx.y];
  const int k0 = k * B;
  const int j0 = k0 + B * (1 + blockIdx.x);
  if (j0 >= d.n || (d.bw > 0 && (int)blockIdx.x + 1 > d.bw)) return;  // past the end, or a zero tile
  const int nb = min(B, d.n - k0), nc = min(B, d.n - j0);
  load_tile(D, d.dinv + (size_t)k * B * B, B, B, B);
  load_tile(Bt, d.R + k0 + (size_t)j0 * d.ld, d.ld, nb, nc);
  __syncthreads();
  apply_inv_tile(D, Bt, nb);
  store_tile(Bt, d.R + k0 + (size_t)j0 * d.ld, d.ld, nb, nc);
  pdl_trigger();
}

// Tile step k, phase 3: A_ij -= U_ki^T U_kj for k < i <= j (upper trailing tiles).
template <typename T, int B = TB>
__global__ void __launch_bounds__(TileGeom<B>::NTH) k_potrf_update(const RowDesc<T>* __restrict__ rows, int k) {
  __shared__ TileSmemB<T, B> sm;
  pdl_wait();
  const RowDesc<T> d = rows[blockIdx.y];
  const int nt = (d.n + B - 1) / B;
  const int m = nt - k - 1;  // trailing tiles per side
  if (m <= 0) return;
  int lin = blockIdx.x;
  if (lin >= m * (m + 1) / 2) return;
  // decode lin -> (i, j) with i <= j, row-wise over the upper triangle
  int i = 0;
  while (lin >= m - i) { lin -= m - i; ++i; }
  const int j = i + lin;
  if (d.bw > 0 && j + 1 > d.bw) return;  // U_kj is a zero tile: nothing to subtract
  const int i0 = (k + 1 + i) * B, j0 = (k + 1 + j) * B, k0 = k * B;
  const int mi = min(B, d.n - i0), nj = min(B, d.n - j0), kb = min(B, d.n - k0);
  T acc[4][TileGeom<B>::CB];
  zero_acc(acc);
  if (i == j)  // diagonal tile: only its upper triangle is used
    tn_acc<T, true, B>(acc, d.R + k0 + (size_t)i0 * d.ld, d.ld, mi, d.R + k0 + (size_t)j0 * d.ld, d.ld, nj, kb, sm);
  else
    tn_acc<T, false, B>(acc, d.R + k0 + (size_t)i0 * d.ld, d.ld, mi, d.R + k0 + (size_t)j0 * d.ld, d.ld, nj, kb, sm);
  sub_store<B>(acc, d.R + i0 + (size_t)j0 * d.ld, d.ld, mi, nj);
  pdl_trigger();
}

// Banded upper Cholesky (Sec. 2.4) of the step-1 pivot blocks, FP64, one
// CTA per block.  A step-1 pivot is the restriction of A to one leaf
// cluster, vertices in increasing id (lexicographic on grids), so its
// nonzeros lie within a half-bandwidth b of the diagonal (b = 49-64 for the
// 7³-8³ leaves of a 3D grid); the Cholesky factor keeps that band, and the
// right-looking elimination touches only the (b + 2)-column window ahead of
// the pivot.  The window lives in shared memory as a ring of b + 2 columns
// (column j at slot j mod (b + 2), its rows j - b .. j); per step two pivot
// rows k, k + 1:
//   1. one thread forms the 2 x 2 pivot block, U_kk = sqrt(A_kk),
//      U_{k,k+1} = A_{k,k+1} / U_kk, U_{k+1,k+1} = sqrt(A_{k+1,k+1} - U_{k,k+1}^2);
//   2. the rows U_k. and U_{k+1,.} across the band, one column per thread;
//   3. the rank-2 update A_ij -= U_ki U_kj + U_{k+1,i} U_{k+1,j} of the
//      b (b + 1) / 2 window entries k + 1 < i <= j <= k + 1 + b, spread evenly
//      over the threads by a table of (i, j) offsets;
//   4. columns k, k + 1 are final: each thread stores its element of them
//      and puts in its place the element of column k + b + 2 (or k + b + 3),
//      which no step has touched yet; the global load is issued before 3
//      and the store after it (3 touches only columns k + 2 and up), so its
//      latency hides behind the update.
// The tiled kernels would do about four times the arithmetic on such a band
// (a 32 x 32 tile step covers rows k .. k + 95 in full).  A pivot that is not
// positive is reported like the tiled kernels' (the block's batch index + 1).
constexpr int BAND_MAX = 96;   // widest band taken by this kernel
constexpr int BAND_NT = 256;   // >= 2 (BAND_MAX + 1): one element of step 4 per thread
static_assert(BAND_NT >= 2 * (BAND_MAX + 1), "one element of step 4 per thread");

template <typename TS>
struct BandTask {
  TS* R;            // the block, column-major, leading dimension ld (upper triangle read and overwritten)
  int32_t n, ld, band, entry;  // entry: index of the block in its pivot batch (for the failure flag)
};

// Column stride of the window: b + 1 entries, rounded up to an even count of
// doubles.  Step 2's threads walk the window diagonally (column + 1, row - 1:
// a stride of one column less one element), which must be odd for the
// threads of a warp to spread over the shared-memory banks.
__host__ __device__ inline int band_cl(int b) { return (b + 2) & ~1; }

__host__ __device__ inline size_t band_smem(int b) {
  return (size_t)(b + 2) * band_cl(b) * sizeof(double) + 2 * (size_t)(b + 2) * sizeof(double) +
         (((size_t)b * (b + 1) / 2 * sizeof(uint16_t) + 15) & ~size_t(15));
}

// TS: the factor's storage type; the block is read from it and U written
// back to it directly (an FP32 factor needs no FP64 copy: the window is
// FP64), all arithmetic in FP64.
template <typename TS>
__global__ void __launch_bounds__(BAND_NT) k_potrf_band(const BandTask<TS>* __restrict__ tasks, int* info) {
  pdl_wait();
  const BandTask<TS> d = tasks[blockIdx.x];
  const int n = d.n, b = d.band, ld = d.ld, tid = threadIdx.x;
  const int WS = b + 2, CL = band_cl(b), CB = b + 1;  // CB: entries used per column
  extern __shared__ __align__(16) unsigned char smraw[];
  double* win = reinterpret_cast<double*>(smraw);
  double* u0 = win + (size_t)WS * CL;  // u0[x] = U(k, k + x), x = 0 .. b + 1
  double* u1 = u0 + WS;                // u1[x] = U(k + 1, k + x)
  uint16_t* pairs = reinterpret_cast<uint16_t*>(u1 + WS);  // (xi << 8) | xj, 2 <= xi <= xj <= b + 1
  __shared__ double sc[4];
  __shared__ int ok;
  const int npairs = b * (b + 1) / 2;
  // pair table: column xj = 2 .. b + 1 holds rows xi = 2 .. xj
  for (int xj = 2 + tid; xj <= b + 1; xj += BAND_NT) {
    int e = (xj - 2) * (xj - 1) / 2;
    for (int xi = 2; xi <= xj; ++xi) pairs[e++] = (uint16_t)((xi << 8) | xj);
  }
  // initial window: columns 0 .. min(n, WS) - 1 into slots 0 ..
  for (int e = tid; e < min(n, WS) * CB; e += BAND_NT) {
    const int j = e / CB, r = e % CB, i = j - b + r;
    win[(size_t)j * CL + r] = i >= 0 ? (double)d.R[i + (size_t)j * ld] : 0.0;
  }
  __syncthreads();
  for (int k = 0; k < n; k += 2) {
    const bool two = k + 1 < n;
    const int k1 = k + 1;
    if (tid == 0) {  // 1. the pivot block
      const double a00 = win[(size_t)(k % WS) * CL + b];
      const double r0 = rsqrt(a00), u00 = a00 * r0;
      const double u01 = two ? win[(size_t)(k1 % WS) * CL + b - 1] * r0 : 0.0;
      const double s11 = two ? win[(size_t)(k1 % WS) * CL + b] - u01 * u01 : 1.0;
      const double r1 = rsqrt(s11), u11 = s11 * r1;
      sc[0] = r0;
      sc[1] = u01;
      sc[2] = r1;
      sc[3] = u11;
      u0[0] = u00;
      ok = (a00 > 0.0) && (s11 > 0.0);
    }
    __syncthreads();
    if (!ok) {
      if (tid == 0) atomicCAS(info, 0, d.entry + 1);
      return;  // uniform
    }
    // 2. rows k and k + 1 of U across the band (x = j - k)
    for (int x = 1 + tid; x <= b + 1; x += BAND_NT) {
      const int j = k + x;
      double v0 = 0.0, v1 = 0.0;
      if (j < n) {
        double* col = win + (size_t)(j % WS) * CL;
        if (x <= b) {
          v0 = col[k - j + b] * sc[0];
          col[k - j + b] = v0;
        }
        if (two) {
          v1 = x == 1 ? sc[3] : (col[k1 - j + b] - sc[1] * v0) * sc[2];
          col[k1 - j + b] = v1;
        }
      }
      u0[x] = v0;
      u1[x] = v1;
    }
    if (tid == 0) win[(size_t)(k % WS) * CL + b] = u0[0];
    __syncthreads();
    // 4. (issued first, it overlaps 3: disjoint columns) columns k, k + 1
    // are final: each thread reads the element of column k + WS or
    // k + 1 + WS it will put in place of its element of column k or k + 1
    const int e4 = tid;  // 2 (b + 1) <= 2 (BAND_MAX + 1) < BAND_NT elements
    const bool has4 = e4 < 2 * CB && k + e4 / CB < n;
    double nv = 0.0;
    int c4 = 0, r4 = 0;
    if (has4) {
      c4 = k + e4 / CB;
      r4 = e4 % CB;
      const int cn = c4 + WS, in = cn - b + r4;
      if (cn < n && in >= 0) nv = (double)d.R[in + (size_t)cn * ld];
    }
    // 3. rank-2 update of the window ahead of the pivot rows
    // (a single last row, n = k + 1, has nothing after it to update)
    if (two)
      for (int e = tid; e < npairs; e += BAND_NT) {
        const int xi = pairs[e] >> 8, xj = pairs[e] & 0xff;
        const int j = k + xj;
        if (j >= n) continue;
        const int i = k + xi;
        double& a = win[(size_t)(j % WS) * CL + (i - j + b)];
        a = fma(-u1[xi], u1[xj], fma(-u0[xi], u0[xj], a));
      }
    if (has4) {
      double* slot = win + (size_t)(c4 % WS) * CL;
      const int i = c4 - b + r4;
      if (i >= 0) d.R[i + (size_t)c4 * ld] = (TS)slot[r4];
      if (c4 + WS < n) slot[r4] = nv;
    }
    __syncthreads();
  }
  pdl_trigger();
}

// The inverses U_kk^{-T} of the 64 x 64 diagonal tiles of a factored pivot
// block (for the block-row solves of k_trsm_cols), tile k = blockIdx.x of
// block blockIdx.y, from U itself (rows and columns beyond n: the identity).
// In 32 x 32 blocks, U^{-1} = [D11, -D11 U12 D22; 0, D22]: each diagonal
// block is inverted by one warp, a lane per column by back substitution in
// registers (no block barrier inside), then the corner by two 32 x 32
// products, four 32 x 32 warps; the result is stored transposed.
constexpr int INV_NT = 128;
template <typename T>
__global__ void __launch_bounds__(INV_NT) k_inv_diag(const RowDesc<T>* __restrict__ rows) {
  extern __shared__ __align__(16) unsigned char smraw[];
  SqTile<T>& U = *reinterpret_cast<SqTile<T>*>(smraw);
  SqTile<T>& D = *reinterpret_cast<SqTile<T>*>(smraw + sizeof(SqTile<T>));  // U^{-1}; its lower-left block: W
  const RowDesc<T> d = rows[blockIdx.y];
  const int k0 = blockIdx.x * TB;
  if (k0 >= d.n) return;
  const int nb = min(TB, d.n - k0);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < TB * TB; e += INV_NT) {
    const int i = e & (TB - 1), j = e / TB;
    U.v[i][j] = (i < nb && j < nb) ? d.R[(k0 + i) + (size_t)(k0 + j) * d.ld] : (i == j ? T(1) : T(0));
  }
  __syncthreads();
  if (warp < 2) {  // D_bb = U_bb^{-1}: column j = lane, rows i <= j
    const int o = 32 * warp, j = lane;
    const T rinv = T(1) / U.v[o + lane][o + lane];
    T x[32];
#pragma unroll
    for (int i = 31; i >= 0; --i) {
      T acc = (i == j) ? T(1) : T(0);
#pragma unroll
      for (int k = i + 1; k < 32; ++k) acc = fma(-U.v[o + i][o + k], x[k], acc);
      const T ri = __shfl_sync(0xffffffffu, rinv, i);
      x[i] = (i > j) ? T(0) : acc * ri;
    }
#pragma unroll
    for (int i = 0; i < 32; ++i) D.v[o + i][o + j] = x[i];
  }
  __syncthreads();
  // W = U12 D22 into D's lower-left block (rows 32.., columns ..31)
  const int jc = lane, i0 = warp;  // thread: column jc, rows i0 + 4 m
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int i = i0 + 4 * m;
    T acc = T(0);
    for (int k = 0; k <= jc; ++k) acc = fma(U.v[i][32 + k], D.v[32 + k][32 + jc], acc);
    D.v[32 + i][jc] = acc;
  }
  __syncthreads();
  // D12 = -D11 W
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int i = i0 + 4 * m;
    T acc = T(0);
    for (int k = i; k < 32; ++k) acc = fma(D.v[i][k], D.v[32 + k][jc], acc);
    D.v[i][32 + jc] = -acc;
  }
  __syncthreads();
  T* out = d.dinv + (size_t)blockIdx.x * TB * TB;  // out(i, j) = U^{-1}(j, i), column-major, zero above
  for (int e = tid; e < TB * TB; e += INV_NT) {
    const int i = e & (TB - 1), j = e / TB;
    out[e] = i >= j ? D.v[j][i] : T(0);
  }
}

// B <- U^{-T} B for one panel of at most 64 columns, left-looking over the
// row tiles (B_i -= sum_{l<i} U_li^T X_l; X_i = U_ii^{-T} B_i).  Rows of B
// above i_start are zero (identity right-hand sides) and are skipped.  The
// next row tile's U_ii^{-T} and B_i (neither written by this tile) are
// copied asynchronously while this tile's GEMM with the solved rows runs.
template <typename T>
__global__ void __launch_bounds__(NT) k_trsm_cols(const TrsmTask<T>* __restrict__ tasks) {
  extern __shared__ __align__(16) unsigned char smraw[];
  SqTile<T>& U = *reinterpret_cast<SqTile<T>*>(smraw);
  SqTile<T>& B = *reinterpret_cast<SqTile<T>*>(smraw + sizeof(SqTile<T>));
  TileSmem<T>& sm = *reinterpret_cast<TileSmem<T>*>(smraw + 2 * sizeof(SqTile<T>));
  const TrsmTask<T> d = tasks[blockIdx.x];
  const int nc = d.nc;
  if (nc <= 0 || d.n <= 0) return;
  T* X = d.B;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int is = (d.i_start / TB) * TB;
  if (is < d.n) {
    load_tile_async(U, d.dinv + (size_t)(is / TB) * TB * TB, TB, TB, TB);  // U_ii^{-T}
    load_tile_async(B, X + is, d.ldb, min(TB, d.n - is), nc);
  }
  for (int i0 = is; i0 < d.n; i0 += TB) {
    const int nb = min(TB, d.n - i0);
    T acc[4][4];
    zero_acc(acc);
    // rows of U's column block i0 above the band are zero tiles
    const int ls = d.bw > 0 ? max(is, i0 - d.bw * TB) : is;
    if (i0 > ls) tn_acc(acc, d.U + ls + (size_t)i0 * d.ldu, d.ldu, nb, X + ls, d.ldb, nc, i0 - ls, sm);
    cp_async_wait_all();  // this tile's U_ii^{-T} and B_i
    __syncthreads();
#pragma unroll
    for (int ii = 0; ii < 4; ++ii)
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        const int r = tx + 16 * ii, c = ty + 16 * jj;
        B.v[r][c] -= acc[ii][jj];
      }
    __syncthreads();
    apply_inv_tile(U, B, nb);
    store_tile(B, X + i0, d.ldb, nb, nc);
    __syncthreads();
    const int i1 = i0 + TB;
    if (i1 < d.n) {
      load_tile_async(U, d.dinv + (size_t)(i1 / TB) * TB * TB, TB, TB, TB);
      load_tile_async(B, X + i1, d.ldb, min(TB, d.n - i1), nc);
    }
  }
}

// ---------------------------------------------------------------- Schur update

// Pull form of A_{ab} -= sum_s X_{as} X_{bs}^T over the separators s adjacent
// to both a and b (Sec. 2.4), one 64x64 output tile per CTA, contributors in a
// fixed order (deterministic, no atomics).  Writes block (a,b) in a's row and
// its transpose (b,a) in b's row.
template <typename T>
__global__ void __launch_bounds__(NT) k_schur(const SchurTile* __restrict__ tiles,
                                             const SchurBlock<T>* __restrict__ blocks,
                                             const SchurContrib<T>* __restrict__ contribs) {
  __shared__ TileSmem<T> sm;
  const SchurTile t = tiles[blockIdx.x];
  const SchurBlock<T> b = blocks[t.block];
  const int mi = min(TB, b.rows - t.i0), nj = min(TB, b.cols - t.j0);
  T acc[4][4];
  zero_acc(acc);
  for (int c = b.cbeg; c < b.cend; ++c) {
    const SchurContrib<T> s = contribs[c];
    if (s.ns <= 0) continue;
    tn_acc(acc, s.Xa + (size_t)t.i0 * s.lds, s.lds, mi, s.Xb + (size_t)t.j0 * s.lds, s.lds, nj, s.ns, sm);
  }
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  // C1 -= acc; the results of 32 tile rows at a time also go through a
  // shared-memory tile, from which C2 = C1^T is written along C2's rows
  // (coalesced) instead of with a stride of ld2 per lane
  // the GEMM buffers are free (tn_acc ends with a block barrier)
  static_assert(sizeof(TileSmem<T>) >= sizeof(T) * 32 * (TB + 1), "staging tile fits in the GEMM buffers");
  T (*tt)[TB + 1] = reinterpret_cast<T (*)[TB + 1]>(&sm);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      const int c = ty + 16 * jj;
#pragma unroll
      for (int ii = 2 * h; ii < 2 * h + 2; ++ii) {
        const int r = tx + 16 * ii;
        if (r >= mi || c >= nj) continue;
        const size_t o1 = (size_t)(t.i0 + r) + (size_t)(t.j0 + c) * b.ld1;
        const T v = b.C1[o1] - acc[ii][jj];
        b.C1[o1] = v;
        tt[r - 32 * h][c] = v;
      }
    }
    if (!b.C2) continue;  // uniform over the CTA
    __syncthreads();
    for (int rr = warp; rr < 32 && 32 * h + rr < mi; rr += NT / 32)
      for (int c = lane; c < nj; c += 32)
        b.C2[(size_t)(t.j0 + c) + (size_t)(t.i0 + 32 * h + rr) * b.ld2] = tt[rr][c];
    __syncthreads();
  }
}

// ---------------------------------------------------------------- two-sided scaling, second side

// Scaling of an adjacent pair p < q (Sec. 2.5), second side: with
// B = U_p^{-T} A_pq (|p| x |q|, the first side's block-row solve) and the
// pivot inverse Y_q = U_q^{-T} (|q| x |q|, lower triangular, zero above the
// diagonal in memory), the scaled block in q's row is
// O = (U_p^{-T} A_pq U_q^{-1})^T = Y_q B^T (|q| x |p|).  One 64 x 64 tile of
// O per CTA (tile list: task, i0, j0); K stops at the tile's last row, past
// which Y_q is zero.
template <typename T>
struct ScaleTask {
  const T* B;  // p's row at q's columns, leading dimension ldb
  const T* Y;  // Y_q, leading dimension nq
  T* O;        // q's row at p's columns, leading dimension ldo
  int32_t ldb, ldo, np, nq;
};

template <typename T>
__global__ void __launch_bounds__(NT) k_scale_gemm(const SchurTile* __restrict__ tiles,
                                                   const ScaleTask<T>* __restrict__ tasks) {
  constexpr int KC2 = 16;
  __shared__ T ys[KC2][TB + 1], bs[KC2][TB + 1];
  const SchurTile tl = tiles[blockIdx.x];
  const ScaleTask<T> d = tasks[tl.block];
  const int i0 = tl.i0, j0 = tl.j0, tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  T acc[4][4];
  zero_acc(acc);
  const int kend = min(d.nq, i0 + TB);
  constexpr int NL = TB * KC2 / NT;  // elements of each operand per thread and chunk
  T ry[NL], rb[NL];
  auto load = [&](int k0) {  // Y(i0 + i, k0 + kk), B(j0 + i, k0 + kk): lanes along i
#pragma unroll
    for (int r = 0; r < NL; ++r) {
      const int e = tid + NT * r, i = e & (TB - 1), k = k0 + e / TB;
      ry[r] = (i0 + i < d.nq && k < kend) ? d.Y[(i0 + i) + (size_t)k * d.nq] : T(0);
      rb[r] = (j0 + i < d.np && k < kend) ? d.B[(j0 + i) + (size_t)k * d.ldb] : T(0);
    }
  };
  if (kend > 0) load(0);
  for (int k0 = 0; k0 < kend; k0 += KC2) {
#pragma unroll
    for (int r = 0; r < NL; ++r) {
      const int e = tid + NT * r;
      ys[e / TB][e & (TB - 1)] = ry[r];
      bs[e / TB][e & (TB - 1)] = rb[r];
    }
    __syncthreads();
    if (k0 + KC2 < kend) load(k0 + KC2);  // the next chunk's loads overlap this chunk's products
#pragma unroll
    for (int kk = 0; kk < KC2; ++kk) {
      T av[4], bv[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        av[q] = ys[kk][tx + 16 * q];
        bv[q] = bs[kk][ty + 16 * q];
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = i0 + tx + 16 * a, j = j0 + ty + 16 * b;
      if (i < d.nq && j < d.np) d.O[i + (size_t)j * d.ldo] = acc[a][b];
    }
}

// ---------------------------------------------------------------- copies

// Block copies in 32 x 32 tiles, one warp per tile: tile g = CP_WARPS
// blockIdx.x + warp belongs to the task i with tptr[i] <= g < tptr[i + 1]
// (tptr: prefix sums of the tasks' tile counts, ntask + 1 entries; every task
// has at least one tile).  cidx[c] is the task holding tile 32 c, and the
// tasks that start after it within g's chunk of 32 tiles are found with one
// ballot over the next 32 entries of tptr (at most 31 start there).  A task's
// tiles run down its rows first.
constexpr int CP_WARPS = 4;
template <typename T>
__global__ void __launch_bounds__(32 * CP_WARPS) k_copy(const int32_t* __restrict__ tptr,
                                                        const int32_t* __restrict__ cidx, int ntask, int32_t ntile,
                                                        const CopyTask<T>* __restrict__ tasks) {
  __shared__ T s[CP_WARPS][32][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int32_t g = (int32_t)blockIdx.x * CP_WARPS + w;
  if (g >= ntile) return;  // uniform over the warp; the warps never synchronise with each other
  int i = cidx[g >> 5];
  const int j = i + 1 + lane;
  i += __popc(__ballot_sync(0xffffffffu, j < ntask && tptr[j] <= g));
  const CopyTask<T> d = tasks[i];
  const int32_t local = g - tptr[i], nr = (d.rows + 31) >> 5;
  const int r0 = (local % nr) * 32, c0 = (local / nr) * 32;
  const int nc = min(32, d.cols - c0);
  if (!d.trans) {
    const int rr = r0 + lane;
    if (rr < d.rows) {
#pragma unroll 8
      for (int c = 0; c < nc; ++c) d.dst[rr + (size_t)(c0 + c) * d.ldd] = d.src[rr + (size_t)(c0 + c) * d.lds];
    }
    return;
  }
  // dst (rows x cols) = transpose of src (cols x rows): lanes along src's
  // rows (dst's columns) on the way in, along dst's rows on the way out
  const int nrr = min(32, d.rows - r0);
#pragma unroll 8
  for (int c = 0; c < nrr; ++c)
    if (lane < nc) s[w][c][lane] = d.src[(c0 + lane) + (size_t)(r0 + c) * d.lds];
  __syncwarp();
  if (lane < nrr) {
#pragma unroll 8
    for (int c = 0; c < nc; ++c) d.dst[(r0 + lane) + (size_t)(c0 + c) * d.ldd] = s[w][lane][c];
  }
}

// ---------------------------------------------------------------- FP64 pivots of FP32 factors
//
// In the mixed forms the factor is stored in FP32, but the Cholesky of every
// pivot block (eliminated separators, Sec. 2.4, and scaled interfaces,
// Sec. 2.5) runs in FP64: the block is widened into an FP64 copy, factored
// there by the FP64 tile kernels above, and its upper factor U and the
// inverses of U's diagonal tiles are rounded back to FP32 for the FP32 tile
// solves and GEMMs that follow.

struct PivotCopy {
  float* R;           // FP32 diagonal block (leading dimension ld)
  double* W;          // FP64 copy, n x n, leading dimension n
  int32_t n, ld;
};

// W <- (double) R (every entry of the n x n block).
__global__ void k_widen_pivot(const PivotCopy* __restrict__ cps) {
  const PivotCopy c = cps[blockIdx.y];
  const int64_t tot = (int64_t)c.n * c.n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % c.n), j = (int)(e / c.n);
    c.W[e] = (double)c.R[i + (size_t)j * c.ld];
  }
}

// R's upper triangle <- (float) U.
__global__ void k_narrow_pivot(const PivotCopy* __restrict__ cps) {
  const PivotCopy c = cps[blockIdx.y];
  const int64_t tot = (int64_t)c.n * c.n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % c.n), j = (int)(e / c.n);
    if (i <= j) c.R[i + (size_t)j * c.ld] = (float)c.W[e];
  }
}

// Diagonal block <- identity (after scaling, Sec. 2.5: S_p A S_p^T has I on p).
template <typename T>
__global__ void k_set_identity(const RowDesc<T>* __restrict__ rows, int nrows) {
  const RowDesc<T> d = rows[blockIdx.y];
  const int64_t tot = (int64_t)d.n * d.n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % d.n), j = (int)(e / d.n);
    d.R[i + (size_t)j * d.ld] = (i == j) ? T(1) : T(0);
  }
}

}  // namespace spand

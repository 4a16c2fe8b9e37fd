// Counter-based Gaussian test matrices for randomized compression (the
// randomized alternative to the column-pivoted QR named in Sec. 2.6.2): every
// entry is a pure function of (seed, step, cluster, row, column), so any
// kernel can draw any entry without state or communication.
//
// Generator: Philox4x64 with 10 rounds (Salmon, Moraes, Dror and Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC 2011): per round the
// 128-bit products M0 x0 and M1 x2 give x <- (hi1 ^ x1 ^ k0, lo1,
// hi0 ^ x3 ^ k1, lo0), and the key advances by the Weyl constants between
// rounds.  Key (seed, step * 2^32 + cluster); counter (column j, row block
// b = i / 4, 0, 0).  The four words w of a block give uniforms
// u = ((w >> 11) + 1/2) 2^-53 in (0, 1) and, by Box-Muller, rows 4b..4b+3:
// sqrt(-2 ln u0) (cos 2 pi u1, sin 2 pi u1), then the same for (u2, u3).
#pragma once

#include <cstdint>

namespace spand {

__device__ __forceinline__ void philox4x64_10(uint64_t x[4], uint64_t k0, uint64_t k1) {
  constexpr uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  constexpr uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += W0;
      k1 += W1;
    }
    const uint64_t h0 = __umul64hi(M0, x[0]), l0 = M0 * x[0];
    const uint64_t h1 = __umul64hi(M1, x[2]), l1 = M1 * x[2];
    const uint64_t y0 = h1 ^ x[1] ^ k0, y2 = h0 ^ x[3] ^ k1;
    x[0] = y0;
    x[1] = l1;
    x[2] = y2;
    x[3] = l0;
  }
}

// The four Gaussian entries of rows 4b .. 4b + 3 of column j.
__device__ __forceinline__ void philox_gauss4(uint64_t k0, uint64_t k1, uint64_t j, uint64_t b, double z[4]) {
  uint64_t x[4] = {j, b, 0ull, 0ull};
  philox4x64_10(x, k0, k1);
  double u[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) u[k] = ((double)(x[k] >> 11) + 0.5) * 0x1.0p-53;
  const double ra = sqrt(-2.0 * log(u[0])), rb = sqrt(-2.0 * log(u[2]));
  z[0] = ra * cospi(2.0 * u[1]);
  z[1] = ra * sinpi(2.0 * u[1]);
  z[2] = rb * cospi(2.0 * u[3]);
  z[3] = rb * sinpi(2.0 * u[3]);
}

// The same four entries from the same Philox words with Box-Muller in FP32
// (for FP32 sketches): u = (w >> 11) 2^-53 + 2^-54 rounded to float, then
// CUDA's logf / sqrtf / cospif / sinpif; within about 1e-6 of
// philox_gauss4's entries.
__device__ __forceinline__ void philox_gauss4f(uint64_t k0, uint64_t k1, uint64_t j, uint64_t b, float z[4]) {
  uint64_t x[4] = {j, b, 0ull, 0ull};
  philox4x64_10(x, k0, k1);
  float u[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) u[k] = fmaf(__ull2float_rn(x[k] >> 11), 0x1.0p-53f, 0x1.0p-54f);
  const float ra = sqrtf(-2.0f * logf(u[0])), rb = sqrtf(-2.0f * logf(u[2]));
  z[0] = ra * cospif(2.0f * u[1]);
  z[1] = ra * sinpif(2.0f * u[1]);
  z[2] = rb * cospif(2.0f * u[3]);
  z[3] = rb * sinpif(2.0f * u[3]);
}

// out: m x ell, column-major (leading dimension m); one thread per 4-row block
// of one column (grid-stride).
__global__ void k_sketch_philox(uint64_t k0, uint64_t k1, int m, int ell, double* __restrict__ out) {
  const int nb = (m + 3) / 4;
  const int64_t total = (int64_t)nb * ell;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(t / nb), b = (int)(t % nb);
    double z[4];
    philox_gauss4(k0, k1, (uint64_t)j, (uint64_t)b, z);
    double* col = out + (size_t)j * m;
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (4 * b + k < m) col[4 * b + k] = z[k];
  }
}

}  // namespace spand

// Schur update of the elimination (Sec. 2.4) on the 5th-generation tensor
// cores, for FP32 factors with TF32 (kind::tf32) or BF16 (kind::f16) operands
// and FP32 accumulation:  A_{ab} -= sum_s X_{as} X_{bs}^T  (pull form: one
// output tile per CTA, contributors in a fixed order, no atomics).
//
// GB300 mapping: a 128 x 64 output tile per CTA of 128 threads; the
// accumulator lives in 64 TMEM columns (lane = tile row).  The K dimension
// (the separator size of every contributor, concatenated) is cut into chunks
// of 128 bytes per row (32 TF32 or 64 BF16 elements), staged in shared memory
// in the 128-byte-swizzled K-major layout (8-row atoms of 1024 bytes, 16-byte
// chunk c of row r stored at chunk c ^ (r mod 8)), so that the 8 lanes that
// store one row's 128 bytes hit distinct bank groups.  Two stages: while the
// tensor core works on one, the threads store the next chunk, which they
// loaded into registers (16-byte vectors, consecutive lanes along K) during
// the previous MMAs.  One
// elected thread issues 4 MMAs (K = 32 bytes each) per chunk and commits them
// to the stage's mbarrier; every wait on it is bounded.
#pragma once

#include <cuda_bf16.h>

#include <type_traits>

#include "factor_kernels.cuh"

namespace spand {

constexpr int TC_M = 128, TC_N = 64, TC_NT = 128;
constexpr int TC_STAGE_BYTES = (TC_M + TC_N) * 128;          // A and B of one chunk
constexpr int TC_SMEM = 2 * TC_STAGE_BYTES + 1024;           // two stages + alignment slack
constexpr long long kTcWaitCycles = 1ll << 31;               // about a second

__device__ __forceinline__ unsigned tc_smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), leading byte offset unused (16).
__device__ __forceinline__ uint64_t tc_desc_sw128(unsigned saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)(16 >> 4) << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of this architecture family
  d |= (uint64_t)2 << 61;  // 128-byte swizzle
  return d;
}

__device__ __forceinline__ bool tc_wait(unsigned bar, unsigned parity) {
  const long long t0 = clock64();
  for (;;) {
    unsigned ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    if (ok) return true;
    if (clock64() - t0 > kTcWaitCycles) return false;
  }
}

template <bool BF16>
__global__ void __launch_bounds__(TC_NT, 4) k_schur_tc(const SchurTile* __restrict__ tiles,
                                                       const SchurBlock<float>* __restrict__ blocks,
                                                       const SchurContrib<float>* __restrict__ contribs,
                                                       int* __restrict__ timeout_flag) {
  constexpr int BK = BF16 ? 64 : 32;  // K elements per 128-byte row
  constexpr unsigned IDESC = (1u << 4) | ((BF16 ? 1u : 2u) << 7) | ((BF16 ? 1u : 2u) << 10) |
                             ((unsigned)(TC_N >> 3) << 17) | ((unsigned)(TC_M >> 4) << 24);
  extern __shared__ unsigned char tc_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)tc_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) unsigned long long bar[2];
  __shared__ unsigned tslot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const SchurTile t = tiles[blockIdx.x];
  const SchurBlock<float> b = blocks[t.block];
  const int mi = min(TC_M, b.rows - t.i0), nj = min(TC_N, b.cols - t.j0);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(tc_smem_addr(&tslot)),
                 "r"(TC_N) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(tc_smem_addr(&bar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(tc_smem_addr(&bar[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = tslot;

  // the chunk sequence: contributors in order, K in steps of BK
  int ci = b.cbeg, k0 = 0;
  while (ci < b.cend && contribs[ci].ns <= 0) ++ci;
  // prefetch registers, 16 bytes of X per lane (the block rows' leading
  // dimensions are whole 16-byte vectors, and their padding rows are zero, so
  // a vector that starts below ns may run into the padding).  TF32: A holds
  // 128 rows x 8 vectors (thread: row e >> 3, vector e & 7 for e = tid + 128 j),
  // B 64 rows x 8.  BF16: A 128 rows x 16 vectors (row e >> 4, vector e & 15),
  // converted to 4 BF16 values (8 bytes) at load time, B 64 rows x 16.
  constexpr int VPR = BF16 ? 16 : 8;             // 16-byte source vectors per row
  constexpr int NA = TC_M * VPR / TC_NT, NB = TC_N * VPR / TC_NT;
  typedef typename std::conditional<BF16, uint2, uint4>::type Reg;
  Reg ra[NA], rb[NB];
  auto load = [&](int c, int kk) {
    const SchurContrib<float> s = contribs[c];
    auto one = [&](const float* X, int r0, int nr, int e) -> Reg {
      const int row = e / VPR, v = e % VPR, k = kk + 4 * v;
      float4 f = make_float4(0.f, 0.f, 0.f, 0.f);
      if (row < nr && k < s.ns) f = *reinterpret_cast<const float4*>(X + (size_t)(r0 + row) * s.lds + k);
      if constexpr (BF16) {
        __nv_bfloat162 lo = __floats2bfloat162_rn(f.x, f.y), hi = __floats2bfloat162_rn(f.z, f.w);
        return make_uint2(*reinterpret_cast<uint32_t*>(&lo), *reinterpret_cast<uint32_t*>(&hi));
      } else {
        return make_uint4(__float_as_uint(f.x), __float_as_uint(f.y), __float_as_uint(f.z), __float_as_uint(f.w));
      }
    };
#pragma unroll
    for (int j = 0; j < NA; ++j) ra[j] = one(s.Xa, t.i0, mi, tid + TC_NT * j);
#pragma unroll
    for (int j = 0; j < NB; ++j) rb[j] = one(s.Xb, t.j0, nj, tid + TC_NT * j);
  };
  // store of one register vector: 16 bytes (TF32) or 8 bytes (BF16) of row
  // `row` at byte 16 v (TF32) / 8 v (BF16) of the row's 128 bytes
  auto put = [&](unsigned char* base, int e, const Reg& x) {
    const int row = e / VPR, v = e % VPR;
    const int kb = BF16 ? 8 * v : 16 * v;
    *reinterpret_cast<Reg*>(base + (row >> 3) * 1024 + (row & 7) * 128 + ((((kb >> 4) ^ (row & 7))) << 4) +
                            (kb & 15)) = x;
  };
  bool ok = true;
  int it = 0;
  if (ci < b.cend) {
    load(ci, k0);
    for (;;) {
      const int st = it & 1;
      unsigned char* sA = sm + st * TC_STAGE_BYTES;
      unsigned char* sB = sA + TC_M * 128;
      // the stage is free once the MMAs of chunk it - 2 have completed
      const bool late = it >= 2 && !tc_wait(tc_smem_addr(&bar[st]), (unsigned)((it - 2) >> 1) & 1u);
      if (!late) {
#pragma unroll
        for (int j = 0; j < NA; ++j) put(sA, tid + TC_NT * j, ra[j]);
#pragma unroll
        for (int j = 0; j < NB; ++j) put(sB, tid + TC_NT * j, rb[j]);
      }
      // the next chunk into registers while the tensor core runs this one
      k0 += BK;
      if (k0 >= contribs[ci].ns) {
        k0 = 0;
        ++ci;
        while (ci < b.cend && contribs[ci].ns <= 0) ++ci;
      }
      const bool more = ci < b.cend;
      if (more) load(ci, k0);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      if (__syncthreads_or(late)) {  // uniform: a wait that gave up ends the tile
        ok = false;
        break;
      }
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const unsigned a0 = tc_smem_addr(sA), b0 = tc_smem_addr(sB);
#pragma unroll
        for (int s = 0; s < 4; ++s) {  // 32 bytes of K per instruction
          const uint64_t da = tc_desc_sw128(a0 + 32 * s), db = tc_desc_sw128(b0 + 32 * s);
          const unsigned acc = (it > 0 || s > 0) ? 1u : 0u;
          if (BF16)
            asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                         :: "r"(tmem), "l"(da), "l"(db), "r"(IDESC), "r"(acc) : "memory");
          else
            asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
                         :: "r"(tmem), "l"(da), "l"(db), "r"(IDESC), "r"(acc) : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::
                         "r"(tc_smem_addr(&bar[st])) : "memory");
      }
      ++it;
      if (!more) break;
    }
    // the last commit completes after every earlier MMA; on a give-up too the
    // MMAs already issued must finish (bounded wait) before TMEM is freed
    if (it > 0 && !tc_wait(tc_smem_addr(&bar[(it - 1) & 1]), (unsigned)((it - 1) >> 1) & 1u)) ok = false;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  if (__syncthreads_or(!ok)) {
    if (tid == 0) atomicExch(timeout_flag, 1);
  } else {
    // C1 -= acc, lane = tile row, 16 columns per TMEM load (coalesced along
    // C1's rows); the results also go to a shared-memory tile (row stride 65
    // floats) from which C2 = C1^T is written with lanes along C2's rows
    float* T = reinterpret_cast<float*>(sm);  // the stages are free: every MMA has completed
    const int row = 32 * warp + lane;
#pragma unroll
    for (int c0 = 0; c0 < TC_N; c0 += 16) {
      uint32_t r[16];
      if (it > 0) {
        const unsigned ta = tmem + ((unsigned)(32 * warp) << 16) + (unsigned)c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(ta) : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) r[j] = 0u;
      }
      if (row < mi) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int col = c0 + j;
          if (col >= nj) break;
          const size_t o1 = (size_t)(t.i0 + row) + (size_t)(t.j0 + col) * b.ld1;
          const float v = b.C1[o1] - __uint_as_float(r[j]);
          b.C1[o1] = v;
          T[row * (TC_N + 1) + col] = v;
        }
      }
    }
    if (b.C2) {
      __syncthreads();
      for (int rr = warp; rr < mi; rr += TC_NT / 32)
        for (int col = lane; col < nj; col += 32)
          b.C2[(size_t)(t.j0 + col) + (size_t)(t.i0 + rr) * b.ld2] = T[rr * (TC_N + 1) + col];
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TC_N) : "memory");
}


}  // namespace spand

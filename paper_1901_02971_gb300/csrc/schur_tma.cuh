// Schur update of the elimination (Sec. 2.4) on the 5th-generation tensor
// cores with TF32 operands and FP32 accumulation, fed by the tensor memory
// accelerator:  A_{ab} -= sum_s X_{as} X_{bs}^T  (pull form: one 128 x 64
// output tile per CTA, contributors in a fixed order, no atomics).
//
// Operands.  The block row of an eliminated separator s, [U_s | X^T], is a
// column-major |s| x W_s matrix whose columns are contiguous in the
// separator's dofs -- the K dimension of the update.  One 2D tensor map per
// separator row (inner dimension |s|, outer W_s, 128-byte swizzle) serves as
// both operands: a box of 32 K-values x 128 columns starting at the column
// of a (x = k0, y = col_a + i0) is the A chunk, a box of 32 x 64 at the
// column of b the B chunk, landing in shared memory already in the K-major
// 128-byte-swizzled layout of the MMA descriptors.  K beyond |s| is filled
// with zeros by the copy engine; rows past the target block read other
// columns of the row (or zeros past W_s) and only reach accumulator rows that
// are never stored.
//
// Pipeline (128 threads): lane 0 of warp 0 issues the copies of chunk it
// into stage it mod 2 once the MMAs of chunk it - 2 have released it
// (mbarrier `empty`), arming the stage's `full` barrier with the byte count;
// lane 0 of warp 1 waits on `full`, issues four K = 8 MMAs into the TMEM
// accumulator and commits them to `empty`; after the last chunk it commits
// to `done`, on which all four warps wait before reading the accumulator
// (lane = tile row) for the epilogue.  Every wait is bounded; a wait that
// runs out sets the tile's timeout flag, and the CTA still waits (bounded)
// for its issued copies and MMAs before it frees TMEM and leaves.
#pragma once

#include <cuda.h>

#include "schur_tc.cuh"

namespace spand {

constexpr int TM_STAGES = 2;  // 2 x 24 KB: four CTAs per SM (measured: 2 / 3 / 4 stages 1.41 / 1.69 / 2.32 ms)
constexpr int TM_A_BYTES = TC_M * 128, TM_B_BYTES = TC_N * 128;
constexpr int TM_STAGE_BYTES = TM_A_BYTES + TM_B_BYTES;
constexpr int TM_SMEM = TM_STAGES * TM_STAGE_BYTES + 1024;  // stages + alignment slack

struct SchurContribTma {  // one eliminated separator s adjacent to both a and b
  const CUtensorMap* map_a;  // box 32 x 128 over s's block row
  const CUtensorMap* map_b;  // box 32 x 64 over the same row
  int32_t col_a, col_b;      // first column of a's (b's) block X^T in s's row
  int32_t ns, pad;
};

__device__ __forceinline__ void tm_expect(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tm_load(unsigned dst, const CUtensorMap* map, int x, int y, unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      :: "r"(dst), "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar) : "memory");
}

__global__ void __launch_bounds__(TC_NT, 4) k_schur_tma(const SchurTile* __restrict__ tiles,
                                                        const SchurBlock<float>* __restrict__ blocks,
                                                        const SchurContribTma* __restrict__ contribs,
                                                        int* __restrict__ timeout_flag) {
  constexpr unsigned IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(TC_N >> 3) << 17) |
                             ((unsigned)(TC_M >> 4) << 24);
  extern __shared__ unsigned char tm_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)tm_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) unsigned long long full[TM_STAGES], empty[TM_STAGES], done;
  __shared__ unsigned tslot;
  __shared__ int fail;
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
    for (int s = 0; s < TM_STAGES; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(tc_smem_addr(&full[s])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(tc_smem_addr(&empty[s])) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(tc_smem_addr(&done)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fail = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = tslot;
  // chunks: contributors in order (empty ones skipped), K in steps of 32
  int nch = 0;
  for (int c = b.cbeg; c < b.cend; ++c) {
    const int ns = contribs[c].ns;
    if (ns > 0) nch += (ns + 31) >> 5;
  }
  const unsigned sbase = tc_smem_addr(sm);
  if (warp == 0 && lane == 0 && nch > 0) {  // ---- producer: the copy engine fills the stages
    int c = b.cbeg, k0 = 0;
    while (contribs[c].ns <= 0) ++c;
    int it = 0;
    for (; it < nch; ++it) {
      const int st = it % TM_STAGES, use = it / TM_STAGES;
      if (use > 0 && !tc_wait(tc_smem_addr(&empty[st]), (unsigned)(use - 1) & 1u)) {
        atomicExch(&fail, 1);
        break;
      }
      const SchurContribTma s = contribs[c];
      const unsigned fb = tc_smem_addr(&full[st]);
      const unsigned da = sbase + st * TM_STAGE_BYTES, db = da + TM_A_BYTES;
      tm_expect(fb, TM_STAGE_BYTES);
      tm_load(da, s.map_a, k0, s.col_a + t.i0, fb);
      tm_load(db, s.map_b, k0, s.col_b + t.j0, fb);
      k0 += 32;
      if (k0 >= s.ns) {
        k0 = 0;
        ++c;
        while (c < b.cend && contribs[c].ns <= 0) ++c;
      }
    }
    // every issued copy must land before the CTA may leave: wait for the
    // last use of every stage (already complete on the normal path)
    for (int j = max(0, it - TM_STAGES); j < it; ++j)
      if (!tc_wait(tc_smem_addr(&full[j % TM_STAGES]), (unsigned)(j / TM_STAGES) & 1u)) atomicExch(&fail, 1);
  } else if (warp == 1 && lane == 0 && nch > 0) {  // ---- MMA issuer
    for (int it = 0; it < nch; ++it) {
      const int st = it % TM_STAGES, use = it / TM_STAGES;
      if (!tc_wait(tc_smem_addr(&full[st]), (unsigned)use & 1u)) {
        atomicExch(&fail, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const unsigned a0 = sbase + st * TM_STAGE_BYTES, b0 = a0 + TM_A_BYTES;
#pragma unroll
      for (int k = 0; k < 4; ++k) {  // 32 bytes of K per instruction
        const uint64_t da = tc_desc_sw128(a0 + 32 * k), db = tc_desc_sw128(b0 + 32 * k);
        const unsigned acc = (it > 0 || k > 0) ? 1u : 0u;
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
                     :: "r"(tmem), "l"(da), "l"(db), "r"(IDESC), "r"(acc) : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::
                       "r"(tc_smem_addr(&empty[st])) : "memory");
    }
    // completes once every MMA issued above has (also on a give-up)
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::
                     "r"(tc_smem_addr(&done)) : "memory");
  }
  __syncwarp();
  bool ok = true;
  if (nch > 0) ok = tc_wait(tc_smem_addr(&done), 0u);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  if (!ok || fail) {
    if (tid == 0) atomicExch(timeout_flag, 1);
  } else {
    // C1 -= acc, lane = tile row, 16 columns per TMEM load; the results also
    // go to a shared-memory tile (row stride 65 floats, in the stages, all of
    // whose copies and MMAs have completed) from which C2 = C1^T is written
    // with lanes along C2's rows
    float* T = reinterpret_cast<float*>(sm);
    const int row = 32 * warp + lane;
#pragma unroll
    for (int c0 = 0; c0 < TC_N; c0 += 16) {
      uint32_t r[16];
      if (nch > 0) {
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

// umma.cuh -- the 5th-generation tensor core (tcgen05) for sm_103a: shared-memory matrix
// descriptors, instruction descriptors, tensor-memory (TMEM) allocation, MMA issue and
// completion, and TMEM loads.  Inline PTX only.
//
// Use (one CTA, cta_group::1): one warp allocates TMEM columns and writes their base
// address to shared memory; threads write the operand tiles into shared memory, make them
// visible to the asynchronous proxy (fence_proxy_async), synchronise (with tc_fence_before
// / tc_fence_after around the barrier); one thread issues the MMAs and commits them to an
// mbarrier, which every thread waits on; each warp then reads the accumulator rows of its
// own quarter of the TMEM lanes (warp w: lanes 32w .. 32w + 31).  The allocating warp frees
// the columns before the CTA exits.
//
// Operand tiles are K-major without swizzling: the canonical layout of 8 x 8 "core
// matrices" of 16-bit elements, each 128 contiguous bytes (row r at byte 16 r, element k at
// byte 2 k); core matrices adjacent along K are 128 bytes apart (the descriptor's leading
// byte offset), groups of 8 rows are 16 K bytes apart (its stride byte offset).  One
// kind::f16 MMA consumes K = 16, i.e. two core matrices along K, so the k-th step of a
// longer K starts 256 k bytes into the tile.
#pragma once
#include <cstdint>

#include "tma.cuh"

namespace moss {

// byte offset of element (row, k) of a K-major canonical tile with K columns
__host__ __device__ constexpr uint32_t kmaj_off(int row, int k, int K) {
  return (uint32_t)((row >> 3) * (K * 16) + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// shared-memory matrix descriptor of such a tile starting at shared address saddr (16-byte
// aligned): start address, leading byte offset 128, stride byte offset 16 K (all in 16-byte
// units), descriptor version 1, base offset 0, no swizzling
__device__ __forceinline__ uint64_t kmaj_desc(uint32_t saddr, int K) {
  const uint64_t start = (saddr >> 4) & 0x3FFFu;
  const uint64_t lbo = 128u >> 4;
  const uint64_t sbo = ((uint64_t)K * 16u) >> 4;
  return start | (lbo << 16) | (sbo << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16 with BF16 A and B (both K-major), FP32 accumulator,
// dense, M x N (M = 128: one accumulator row per TMEM lane; N a multiple of 16 up to 256)
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4)                        // D format: F32
         | (1u << 7) | (1u << 10)         // A, B format: BF16
         | ((uint32_t)(N >> 3) << 17)     // N / 8
         | ((uint32_t)(M >> 4) << 24);    // M / 16
}

// D (TMEM, at address d) = A B^T (+ D if acc): A given by descriptor a (M x K), B by
// descriptor b (N x K); issued by one thread
__device__ __forceinline__ void umma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, int acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// the barrier's arrival once every MMA this thread issued before has completed
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// barrier initialisation visible to the asynchronous proxy (the MMA's commits)
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// ncols TMEM columns (a power of 2, 32..512) for this CTA; base address written to *dst.
// Executed by all threads of one warp.
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, int ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

// free them (the allocating warp, all threads)
__device__ __forceinline__ void tmem_dealloc(uint32_t base, int ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(ncols) : "memory");
}

// order tcgen05 operations before / after a thread synchronisation
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive FP32 columns of the calling thread's TMEM lane, from address taddr (lane
// field = the warp's first lane); the whole warp executes it
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

}  // namespace moss

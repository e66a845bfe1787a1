// tma.cuh -- bulk asynchronous copies (TMA, cp.async.bulk) from global into shared memory,
// completed on a shared-memory mbarrier, for sm_103a.  Inline PTX only.
//
// Use: one thread initialises the barrier (mbar_init) and, per fill, announces the bytes
// it will bring (mbar_expect_tx) and issues the copies (tma_load_1d); every thread then
// waits for the barrier's phase (mbar_wait).  A copy needs a 16-byte aligned source and
// destination and a size that is a multiple of 16 bytes.
#pragma once
#include <cstdint>

namespace moss {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// make barrier initialisation and earlier shared-memory accesses of this thread visible to
// the asynchronous (TMA) proxy
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// this thread's arrival on the barrier, announcing bytes that copies will complete
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// bytes from global src to shared dst, completing on bar
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the barrier phase with the given parity to complete, at most `limit` polls
// (each poll may suspend the thread for a short, hardware-chosen time).  Returns false if
// the limit was reached.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, unsigned limit) {
  for (unsigned k = 0; k < limit; ++k)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

}  // namespace moss

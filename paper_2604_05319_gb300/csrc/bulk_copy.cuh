// One-dimensional bulk copies global -> shared memory on the copy engine of
// the SM (cp.async.bulk, completion counted on an mbarrier), with a bounded
// wait.  Used to stage a frozen chunk inverse into shared memory while the
// CTA computes the chunk's far field.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hk {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// One thread initialises the barrier (one arrival per phase: the issuing
// thread's arrive.expect_tx), then the CTA synchronises.
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Issued by one thread: bytes (a multiple of 16; both addresses 16-byte
// aligned) from src to dst, completing the barrier's current phase.  The
// fence orders the CTA's earlier generic accesses of dst (made before the
// preceding __syncthreads) before the copy's writes.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Wait for the barrier phase with parity `parity`; gives up after `limit`
// polls (each may suspend the thread for a short, system-dependent time) and
// returns false then.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int limit) {
  for (int i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

}  // namespace hk

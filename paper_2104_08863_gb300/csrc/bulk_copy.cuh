// Bulk asynchronous copies (the TMA engine's 1-D form) from global to shared memory, with
// completion counted in bytes on an mbarrier, and a bounded wait on the mbarrier.  Every address
// is 16-byte aligned and every size a multiple of 16 bytes; the callers check this before
// launching.
#pragma once

#include <stdint.h>

namespace pp {

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// An mbarrier that completes a phase on one arrival (plus the bytes that arrival announces).
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's view of earlier generic-proxy accesses to shared memory (its own, and
// those a barrier made visible to it) before its later asynchronous-proxy accesses.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// The single arrival of the current phase, announcing `bytes` to be counted by complete_tx.
// Copies counted on the barrier may be issued before or after it (the byte count may run
// negative in between); the phase completes once both the arrival and all bytes are in.
__device__ __forceinline__ void mbar_arrive_expect(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

// `bytes` from gmem to smem, completion counted on bar (no arrival).
__device__ __forceinline__ void bulk_copy_in(void* smem, const void* gmem, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(smem)),
               "l"(gmem), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

// Thread 0's whole-tile form: fence, arrival with the byte count, and the copy.
__device__ __forceinline__ void bulk_load(void* smem, const void* gmem, unsigned bytes, uint64_t* bar) {
  fence_proxy_async();
  mbar_arrive_expect(bar, bytes);
  bulk_copy_in(smem, gmem, bytes, bar);
}

// Bounded wait for the completion of phase `parity` of bar; false after about two seconds.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  const long long t0 = clock64();
  for (unsigned it = 0; it < (1u << 26); ++it) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > (1LL << 32)) return false;
  }
  return false;
}

}  // namespace pp

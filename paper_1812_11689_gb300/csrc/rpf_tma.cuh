// rpf_tma.cuh -- bulk asynchronous copies (TMA engine, cp.async.bulk) of
// point rows into shared memory, completed on an mbarrier.
//
// A CTA stages up to blockDim rows at once: thread 0 posts the expected byte
// count, every thread then issues the bulk copy of its own row (one 16-byte
// aligned, 16-byte-multiple global span), and all threads wait on the
// barrier's phase.  Every wait is bounded in time: after `limit_ns`
// nanoseconds of the global timer (rpf_set_wait_limit; 2 s by default) the
// thread records RPF_ETIMEOUT in the error word and gives up.
#pragma once

#include "rpf_internal.cuh"

__device__ __forceinline__ uint32_t rpf_smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void rpf_mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(rpf_smem_addr(bar)), "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void rpf_mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(rpf_smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool rpf_mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(rpf_smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t rpf_globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait for the given phase parity: polls until the phase completes or
// limit_ns nanoseconds of the global timer have passed (checked every 64
// polls; at most 2^24 checks in any case).  Returns false and sets *err on
// timeout.
__device__ __forceinline__ bool rpf_mbar_wait(uint64_t* bar, uint32_t parity, int* err,
                                              uint64_t limit_ns) {
  if (rpf_mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = rpf_globaltimer();
  for (uint32_t it = 0; it < (1u << 24); ++it) {
#pragma unroll 1
    for (int p = 0; p < 64; ++p)
      if (rpf_mbar_try_wait(bar, parity)) return true;
    if (rpf_globaltimer() - t0 > limit_ns) break;
  }
  if (err) atomicExch(err, RPF_ETIMEOUT);
  return false;
}

// Order this thread's earlier generic-proxy accesses of shared memory before
// later async-proxy (bulk copy) writes to it.
__device__ __forceinline__ void rpf_fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Bulk copy of `bytes` (a multiple of 16) from global src (16-byte aligned)
// to shared dst (16-byte aligned), completing on bar.
__device__ __forceinline__ void rpf_bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                             uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(rpf_smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(rpf_smem_addr(bar))
      : "memory");
}

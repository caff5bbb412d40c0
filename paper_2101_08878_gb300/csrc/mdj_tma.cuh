// Bulk asynchronous copies (TMA, cp.async.bulk) from global to shared memory
// with mbarrier completion, and bounded waits on them.
//
// Only the 1-D bulk form is used: source and destination 16-byte aligned and
// the size a multiple of 16 bytes.  Callers copy the 16-byte-aligned interior
// of a range and load the unaligned head and tail elements with ordinary
// loads, so no copy reads outside the range.
#pragma once

#include <stdint.h>

namespace mdj {

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Arrive once, announcing `bytes` of transaction count still to land.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Orders this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (bulk copy) accesses.
__device__ __forceinline__ void fence_proxy_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Bulk copy of `bytes` (multiple of 16; both addresses 16-byte aligned) from
// global to shared memory, completing on `bar`.
__device__ __forceinline__ void tma_load_1d(void *dst_smem, const void *src_gmem, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Waits for phase `parity` of `bar` to complete, for at most `limit_ns` of
// device time.  Returns false if the wait ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  for (uint32_t polls = 0; polls < (1u << 26); polls++) {
    if (mbar_try_wait(bar, parity)) return true;
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
  return false;
}

// Plan of a copy of elements [beg, beg + n) of an array of `esize`-byte
// elements at `base` (base 16-byte aligned): the bulk part covers the aligned
// interior [a, b); head elements [beg, a) and tail [b, beg + n) are loaded
// with ordinary loads.  Shared-memory element i of the range lives at index
// (beg - beg_al) + i of a buffer that starts at the aligned-down element
// beg_al (so the bulk part lands on a 16-byte boundary).
struct BulkPlan {
  uint32_t beg_al;   // first element of the buffer (beg rounded down to 16 bytes)
  uint32_t a, b;     // aligned interior [a, b) (element indices)
  uint32_t bytes;    // (b - a) * esize, a multiple of 16
};

__device__ __forceinline__ BulkPlan bulk_plan(uint32_t beg, uint32_t n, uint32_t esize) {
  const uint32_t per = 16 / esize;  // elements per 16 bytes
  BulkPlan p;
  p.beg_al = beg / per * per;
  const uint32_t end = beg + n;
  p.a = (beg + per - 1) / per * per;
  p.b = end / per * per;
  if (p.a > p.b) p.a = p.b = beg;  // range inside one 16-byte chunk: no bulk part
  if (p.b < p.a) p.b = p.a;
  p.bytes = (p.b - p.a) * esize;
  return p;
}

}  // namespace mdj

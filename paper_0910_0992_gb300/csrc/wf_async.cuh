// Asynchronous-copy building blocks for sm_100-class GPUs: mbarriers, bulk global->shared
// copies (cp.async.bulk, completion counted in bytes on an mbarrier), L2 cache-policy
// descriptors, named barriers with an OR reduction, and waits bounded by elapsed device time.
//
// Every wait here gives up after kWaitNs of device time, so a copy that never lands cannot hang
// a kernel: the caller records the failure in an error word, drains what it issued and returns.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace wf {
namespace async {

// a copy normally lands within microseconds; the limit is on elapsed time because how long one
// try_wait may suspend is not specified
constexpr unsigned long long kWaitNs = 500000000ull;

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// order this thread's earlier generic-proxy accesses of shared memory before later bulk copies
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_addr(bar)),
      "r"(bytes)
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for the phase of the given parity. Returns false if kWaitNs passed first, or, when
// `abort` is given, as soon as *abort is non-zero (another thread of the CTA gave up).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, const volatile int* abort = nullptr) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = now_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (abort && *abort) return false;
    if (now_ns() - t0 > kWaitNs) return false;
  }
  return true;
}

// L2 policy descriptors for the cache hints of bulk copies
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// bytes (a multiple of 16) from global src to shared dst, both 16-byte aligned; completion is
// counted on bar (whose expected transaction count the issuing thread has raised)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  unsigned long long gsrc;
  asm volatile("cvta.to.global.u64 %0, %1;" : "=l"(gsrc) : "l"(src));
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
      "l"(gsrc), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// the same with an L2 cache-policy hint
__device__ __forceinline__ void bulk_g2s_hint(void* dst, const void* src, unsigned bytes, uint64_t* bar, uint64_t pol) {
  unsigned long long gsrc;
  asm volatile("cvta.to.global.u64 %0, %1;" : "=l"(gsrc) : "l"(src));
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_addr(dst)),
      "l"(gsrc), "r"(bytes), "r"(smem_addr(bar)), "l"(pol)
      : "memory");
}

// named barrier over `count` threads (a multiple of 32); id 0 is __syncthreads'
__device__ __forceinline__ void named_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// named barrier that also returns the OR of `v` over the participating threads (all of them
// receive the same value, so a decision taken on it is uniform)
__device__ __forceinline__ bool named_sync_or(int id, int count, bool v) {
  unsigned r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.or.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((unsigned)v), "r"(id), "r"(count)
      : "memory");
  return r != 0;
}

}  // namespace async
}  // namespace wf

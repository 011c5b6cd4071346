// mbarrier helpers with bounded waits for the tensor-core kernel: every wait
// gives up after a time limit (measured on %globaltimer), raises the CTA's
// abort flag and records TPIR_ETIMEDOUT in the device status word, so that a
// pipeline that stops making progress ends the kernel instead of hanging it.
#pragma once

#include <cstdint>

#include "../../include/talekpir.h"

namespace tpir {
namespace mb {

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ uint32_t saddr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void arrive(uint64_t* bar) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\tmbarrier.arrive.release.cta.shared::cta.b64 st, [%0];\n\t}" ::"r"(
          saddr(bar))
      : "memory");
}
// The thread sleeps in try_wait until the phase completes or about a
// millisecond passes (the suspend-time hint), instead of spinning.
__device__ __forceinline__ bool try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2, 1000000;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(saddr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Non-blocking test for completion of phase `parity`.
__device__ __forceinline__ bool test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(saddr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for phase `parity` of `bar` to complete; false if the CTA aborted or
// the wait ran past limit_ns (then the abort flag and the status word are set).
__device__ __forceinline__ bool wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                     int* status, uint64_t limit_ns) {
  if (try_wait(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  while (!try_wait(bar, parity)) {
    if (*abort_flag) return false;
    if (gtimer() - t0 > limit_ns) {
      *abort_flag = 1;
      atomicExch(status, static_cast<int>(TPIR_ETIMEDOUT));
      return false;
    }
  }
  return true;
}

// The same wait for phases expected to take long (whole work items): after
// the first failed poll it sleeps between polls, leaving the issue slots to
// the warps that do the work.
__device__ __forceinline__ bool wait_sleep(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                           int* status, uint64_t limit_ns, uint32_t sleep_ns) {
  if (try_wait(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  while (!try_wait(bar, parity)) {
    if (*abort_flag) return false;
    if (gtimer() - t0 > limit_ns) {
      *abort_flag = 1;
      atomicExch(status, static_cast<int>(TPIR_ETIMEDOUT));
      return false;
    }
    __nanosleep(sleep_ns);
  }
  return true;
}

// ---- CTA pairs (clusters of two): barriers that the other CTA arrives at ----
// Address of this CTA's shared variable p in the shared memory of CTA `rank`
// of the cluster.
__device__ __forceinline__ uint32_t cluster_addr(const void* p, uint32_t rank) {
  uint32_t a;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(a) : "r"(saddr(p)), "r"(rank));
  return a;
}
// Arrival, with release at cluster scope, at a barrier given by its cluster
// address (this CTA's own or the other CTA's).
__device__ __forceinline__ void arrive_cluster(uint32_t cluster_bar) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_bar)
               : "memory");
}
__device__ __forceinline__ bool try_wait_cluster(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2, 1000000;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(saddr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// wait() for a barrier that the other CTA of the pair arrives at (acquire at
// cluster scope); bounded the same way.
__device__ __forceinline__ bool wait_cluster(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                             int* status, uint64_t limit_ns) {
  if (try_wait_cluster(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  while (!try_wait_cluster(bar, parity)) {
    if (*abort_flag) return false;
    if (gtimer() - t0 > limit_ns) {
      *abort_flag = 1;
      atomicExch(status, static_cast<int>(TPIR_ETIMEDOUT));
      return false;
    }
  }
  return true;
}
// Both CTAs of the cluster reach this point (all threads of each).
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" :::
                   "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

}  // namespace mb
}  // namespace tpir

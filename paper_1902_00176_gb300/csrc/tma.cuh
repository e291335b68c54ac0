// tma.cuh -- bulk asynchronous copies (the TMA's non-tensor form) with mbarrier
// completion, for kernels that stage whole rows of global memory in shared
// memory. Every wait is bounded: a wait that runs out reports failure and the
// caller records an error code in the plan's device error word and returns.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gfc {

// error codes written to the device error word
constexpr int kErrBulkWait = 0x7401;  // an mbarrier wait for a bulk copy ran out

// a wait for a bulk copy gives up after this long (the copies here take
// microseconds), or after kMbarPolls polls if the global timer does not advance
constexpr unsigned long long kMbarTimeoutNs = 2000000000ull;
constexpr unsigned kMbarPolls = 1u << 28;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// order this thread's earlier generic-proxy accesses of shared memory before
// later async-proxy (bulk copy) writes to it
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

// one thread: expect `bytes` more on the barrier's current phase (one arrival)
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

// start a copy of `bytes` (a multiple of 16; both addresses 16-byte aligned)
// from global to shared memory that completes on `bar`
__device__ __forceinline__ void bulk_copy(void* dst_smem, const void* src_gmem, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_addr(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// L2 eviction policies (createpolicy): data read or written once goes first,
// the spectrum handed from the row pass to the inverse row pass goes last
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;\n" : "=l"(p));
  return p;
}

// bulk_copy with an L2 eviction policy for the lines it reads
__device__ __forceinline__ void bulk_copy_hint(void* dst_smem, const void* src_gmem, unsigned bytes, uint64_t* bar,
                                               uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;\n" ::"r"(
          smem_addr(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
      : "memory");
}

// 8-byte global store with an L2 eviction policy
__device__ __forceinline__ void st_global_hint(float2* p, float2 v, uint64_t policy) {
  asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;\n" ::"l"(p), "f"(v.x), "f"(v.y), "l"(policy)
               : "memory");
}

// Drop the whole 128-byte L2 lines inside [begin, begin + bytes) without
// writing them back (their data is dead: read for the last time). Lines that
// the range only partly covers are left alone. The calling threads split the
// lines by `rank` of `count`.
__device__ __forceinline__ void l2_discard_range(const void* begin, size_t bytes, int rank, int count) {
  const uintptr_t b = reinterpret_cast<uintptr_t>(begin), e = b + bytes;
  const uintptr_t first = (b + 127) & ~(uintptr_t)127, last = e & ~(uintptr_t)127;
  for (uintptr_t a = first + (uintptr_t)rank * 128; a < last; a += (uintptr_t)count * 128)
    asm volatile("discard.global.L2 [%0], 128;\n" ::"l"(a) : "memory");
}

// one thread: expect and start one copy
__device__ __forceinline__ void bulk_load(void* dst_smem, const void* src_gmem, unsigned bytes, uint64_t* bar) {
  mbar_expect_tx(bar, bytes);
  bulk_copy(dst_smem, src_gmem, bytes, bar);
}

// start fetching `bytes` (a multiple of 16) of global memory at a 16-byte
// aligned address into L2; nothing waits for it
__device__ __forceinline__ void l2_prefetch(const void* src_gmem, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(src_gmem), "r"(bytes) : "memory");
}

// one thread: start a copy of `bytes` (a multiple of 16; both addresses 16-byte
// aligned) from shared to global memory, in this thread's current bulk group
__device__ __forceinline__ void bulk_store(void* dst_gmem, const void* src_smem, unsigned bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(dst_gmem),
               "r"(smem_addr(src_smem)), "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
}

// the issuing thread: wait until its bulk stores have read their shared-memory
// sources (the buffer may be written again)
__device__ __forceinline__ void bulk_store_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
}

// the issuing thread: wait until its bulk stores have completed
__device__ __forceinline__ void bulk_store_wait() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }

// wait until the barrier's phase `parity` has completed; false if the time
// bound ran out
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity,
                                          unsigned long long timeout_ns = kMbarTimeoutNs) {
  const unsigned a = smem_addr(bar);
  const unsigned long long t0 = global_ns();
  for (unsigned i = 0; i < kMbarPolls; ++i) {
    unsigned done;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (global_ns() - t0 > timeout_ns) return false;
  }
  return false;
}

}  // namespace gfc

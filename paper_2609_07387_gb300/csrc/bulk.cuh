// Bulk asynchronous copies (the TMA unit's untiled form) between global and
// shared memory, completed on an mbarrier; every wait bounded.
//
// Rules the callers keep: both addresses and the size are multiples of 16
// bytes; one mbarrier phase expects exactly the bytes its copies deliver.
#pragma once

#include <cstdint>

namespace ucns {

constexpr long long kBulkWaitCycles = 1ll << 30;  // ~0.5 s at 2 GHz: a wait gives up after this

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint64_t* bar, uint32_t count = 1) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// one plain arrival (no bytes announced)
__device__ __forceinline__ void bar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// the single arrival of the phase, announcing `bytes` of incoming copies
__device__ __forceinline__ void bar_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

// global -> shared, `bytes` counted on `bar`
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

// bounded wait for the phase with the given parity; false if it gave up
// after `limit` cycles
__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity, long long limit = kBulkWaitCycles) {
  const long long t0 = clock64();
  for (uint32_t it = 0;; it++) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 63u) == 63u && clock64() - t0 > limit) return false;
  }
}

// 16-byte asynchronous copy global -> shared (L2 only), tracked per thread
__device__ __forceinline__ void async_copy16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}

// one arrival on `bar` once this thread's earlier async_copy16 copies have
// landed (the arrival is one of the barrier's expected count)
__device__ __forceinline__ void async_copies_arrive(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// make this thread's generic-proxy shared-memory writes visible to the bulk copy unit
__device__ __forceinline__ void fence_smem_to_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// shared -> global, then wait until the shared source has been read
__device__ __forceinline__ void bulk_store(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src)),
               "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// The give-up path of bar_wait, exercised on its own: one thread waits, with
// a short limit, for a phase of a fresh mbarrier that nothing arrives on and
// no copy completes (nothing is in flight), then reports the timeout as the
// reconstruction does (bit 1 of the error word).
__global__ void k_bulk_wait_probe(int* err, long long limit) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  bar_init(&bar);
  if (!bar_wait(&bar, 0, limit)) atomicOr(err, 2);
}

}  // namespace ucns

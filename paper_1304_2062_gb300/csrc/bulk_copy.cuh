// Bulk asynchronous copies between device memory and shared memory
// (cp.async.bulk, issued by one thread, completion counted in bytes on an
// mbarrier for loads and by bulk groups for stores), with bounded waits.
#pragma once

#include <stdint.h>

namespace se2n {
namespace bulk {

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// one arrival that also expects `bytes` of copies to complete on the barrier
__device__ __forceinline__ void bar_expect(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool bar_try(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity), "r"(1000000u)
        : "memory");
    return done != 0;
}

// Wait for phase `parity` of the barrier; false once about 2 s of SM cycles
// (kWait, longer at lower clocks) have passed without it. Each try_wait may
// suspend the thread in hardware until the phase completes (up to 1 ms), so
// waiting threads take no issue slots.
constexpr long long kWait = 4000000000LL;
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
    if (bar_try(bar, parity)) return true;
    const long long t0 = clock64();
    for (;;) {
        if (bar_try(bar, parity)) return true;
        if (clock64() - t0 > kWait) return false;
    }
}

// bytes (a multiple of 16, both addresses 16-byte aligned) from device to
// shared memory, completing on bar
__device__ __forceinline__ void load(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// bytes from shared to device memory, in the current bulk group
__device__ __forceinline__ void store(void *dst, uint32_t src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(dst), "r"(src), "r"(bytes)
                 : "memory");
}

// close the current bulk group
__device__ __forceinline__ void store_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }

// wait until this thread's bulk groups have read their shared-memory sources
__device__ __forceinline__ void store_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }

// close the current bulk group and wait until every group of this thread has
// completed (its writes performed)
__device__ __forceinline__ void store_commit_wait() {
    asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
    asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
}

// this thread's shared-memory writes, ordered before later bulk copies that
// read them (each writing thread, then a barrier, then the copy)
__device__ __forceinline__ void fence_to_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

}  // namespace bulk
}  // namespace se2n

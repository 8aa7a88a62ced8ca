// rowstage.cuh -- per-warp staging of gathered rows in shared memory.
//
// The level sweeps add, for every contributing neighbour u of a vertex, u's
// masked row (B uint16 counts forward, B FP32 c values backward). Loading
// those rows into registers keeps only a few in flight per warp, and the
// sweep is then bound by L2 latency. Here the lanes that found a
// contributing neighbour each start one bulk asynchronous copy
// (cp.async.bulk, global -> shared) of that row into the warp's stage; the
// copies complete on one mbarrier per warp (transaction count = bytes), so a
// whole round of up to R rows costs one round trip and no registers.
//
// Every wait is bounded: after kWaitNs the wait gives up and the caller sets
// a status flag (the host reports a timeout) and stops staging.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace bcgb {
namespace stage {

// per-warp stage sizes: forward rows (uint16) and backward rows (FP32); the
// backward kernel trades stage depth for a fourth resident block per SM
constexpr uint32_t kFwdStageBytes = 4096;
constexpr uint32_t kBwdStageBytes = 4096;
constexpr uint64_t kWaitNs = 2000000000ull;  // 2 s per wait

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t now_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// One arrival (the issuing lane's expect_tx) per phase.
__device__ __forceinline__ void bar_init(uint64_t *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// Test the phase; while it is incomplete the thread may be suspended for up
// to kSuspendNs (it resumes as soon as the phase completes), so a waiting
// warp does not take issue slots from the others.
constexpr uint32_t kSuspendNs = 20000;
__device__ __forceinline__ bool try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(kSuspendNs)
        : "memory");
    return ok != 0u;
}

// Bounded wait for the phase with the given parity; false once the bound
// passed: limit_us microseconds, or kWaitNs when limit_us is 0.
__device__ __forceinline__ bool wait(uint64_t *bar, uint32_t parity, uint32_t limit_us = 0) {
    if (try_wait(bar, parity)) return true;
    const uint64_t limit_ns = limit_us ? (uint64_t)limit_us * 1000ull : kWaitNs;
    const uint64_t t0 = now_ns();
    while (!try_wait(bar, parity))
        if (now_ns() - t0 > limit_ns) return false;
    return true;
}

// Count `bytes` of the current phase's expected transactions as done without
// a copy (releases bytes that were expected but will not arrive).
__device__ __forceinline__ void complete_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.complete_tx.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

// Bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned)
// from global to shared memory, completing on bar.
__device__ __forceinline__ void copy(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(static_cast<uint64_t>(__cvta_generic_to_global(src))), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Hint: bring `bytes` (a multiple of 16, 16-byte aligned) of global memory
// into L2 without waiting for it.
__device__ __forceinline__ void prefetch_l2(const void *src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(
                     static_cast<uint64_t>(__cvta_generic_to_global(src))),
                 "r"(bytes)
                 : "memory");
}

}  // namespace stage
}  // namespace bcgb

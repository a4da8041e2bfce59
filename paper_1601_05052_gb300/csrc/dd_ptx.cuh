// dd_ptx.cuh -- inline-PTX building blocks for sm_103a: mbarriers, 1-D TMA
// bulk copies (global -> shared) and bounded waits.
//
// Every wait on an mbarrier is bounded by a wall-clock budget read from
// %globaltimer; when it runs out the waiting thread records an error bit in
// the plan's device error word and stops waiting, so a lost copy can never
// hang the GPU.
#pragma once
#include <cstdint>

#include "dd_errbits.h"

namespace dd {

// Budget for one mbarrier wait: 2 s of wall clock. A staging copy normally
// lands in microseconds.
constexpr unsigned long long kWaitBudgetNs = 2000000000ull;

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

// Makes barrier initialisation visible to the async (TMA) proxy.
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Orders this thread's earlier generic-proxy shared-memory accesses (as
// published to it by a CTA barrier) before its later async-proxy writes.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_addr(bar)),
        "r"(bytes)
        : "memory");
}

// Plain arrival (count 1, no transaction bytes).
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_addr(bar))
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

// Bounded wait for the phase with the given parity to complete. Returns false
// (and sets kErrWaitTimeout in *err) if the budget ran out.
//
// `gave_up` (shared memory, nullable) is the CTA's give-up flag: a wait that
// has to spin and finds it set returns false at once, and a wait that runs
// out sets it. Once one hand-off of a CTA is lost its barriers' phases are
// out of step (a later parity test could pass on a stale phase), so later
// waits of the CTA fail fast, the caller skips the work that depended on
// them, and no result of the CTA is stored after the flag is set.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int *err,
                                                  unsigned long long budget_ns = kWaitBudgetNs,
                                                  volatile int *gave_up = nullptr) {
    // A phase that has already completed is taken without reading the flag
    // (the common case costs one try_wait); a CTA that gave up learns it at
    // its next wait that has to spin, and its callers check the flag before
    // storing results.
    if (mbar_try_wait(bar, parity)) return true;
    if (gave_up && *gave_up) return false;
    const unsigned long long t0 = globaltimer_ns();
    for (;;) {
        for (int i = 0; i < 64; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (gave_up && *gave_up) return false;
        if (globaltimer_ns() - t0 > budget_ns) {
            if (err) atomicOr(err, kErrWaitTimeout);
            if (gave_up) *gave_up = 1;
            return false;
        }
    }
}

// 1-D bulk copy global -> shared through the TMA unit, completion counted in
// bytes on `bar`. dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

}  // namespace dd

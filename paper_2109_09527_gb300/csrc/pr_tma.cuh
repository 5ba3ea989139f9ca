// Shared-memory pipelines fed by bulk asynchronous copies (cp.async.bulk, the
// 1-D form of GB300's TMA) with mbarrier completion: the helpers of the
// pipelined synchronous row kernel (k_rows_tma) and the pipelined barrier-free
// kernel.  A producer arrives on a stage's "full" barrier with the byte count
// of its copies, which complete the phase; consumers wait on it, and arrive
// on the stage's "empty" barrier when done.  Every wait is bounded.
#pragma once

#include "pr_tile.cuh"

// L2 eviction priority of the bulk copies (0 = no hint; 1..3 as
// PRK_L2_STREAM): evict_first, so that the streamed column indices do not
// push the gathered quotient vector out of L2.
#ifndef PRK_L2_BULK
#define PRK_L2_BULK 1
#endif

namespace prk {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
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

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait until the phase of `bar` with this parity has completed; false after
// about one second (the bound every device-side wait of the library has).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > 1000000000ull) return false;
    return true;
}

// Bulk copy of `bytes` (a multiple of 16) from global to this block's shared
// memory, both addresses 16-byte aligned, completing on `bar`.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    if constexpr (PRK_L2_BULK == 0) {
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         smem_addr(dst)),
                     "l"(src), "r"(bytes), "r"(smem_addr(bar))
                     : "memory");
    } else {
        // streamed once per iteration: an L2 eviction priority of class PRK_L2_BULK
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], "
            "%4;" ::"r"(smem_addr(dst)),
            "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(l2_policy<PRK_L2_BULK>())
            : "memory");
    }
}

}  // namespace prk

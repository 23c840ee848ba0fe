// Bulk global -> shared copies (the TMA unit's 1D form) completed on an
// mbarrier, for streaming the sorted cells into shared memory ahead of the
// warps that consume them (sm_90 and later; inline PTX).
//
// Use: one thread arms the barrier with the byte count of the copies of one
// phase (arrive + expect_tx), issues the copies, and every consumer waits on
// the phase's parity.  A slot is refilled only after all its readers passed a
// warp barrier; the issuing thread then orders their generic-proxy reads
// before the async-proxy writes with a proxy fence.
#pragma once

#include <cstdint>

namespace dvl {

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// Makes initialised barriers visible to the async proxy (the copy engine).
__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void proxy_fence_shared()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Plain arrival (release at CTA scope): completes the phase of a barrier
// initialised with count 1.
__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// dst (shared), src (global) 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}

// One poll; a thread whose phase is not complete is suspended until it
// completes or `suspend_ns` nanoseconds have passed (so a waiting warp costs
// no issue slots).
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity, uint32_t suspend_ns)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok) : "r"(bar), "r"(parity), "r"(suspend_ns) : "memory");
    return ok != 0;
}

constexpr uint32_t MBAR_SUSPEND_NS = 1000000;   // 1 ms per poll at most

// Waits for the phase with the given parity, at most `limit` polls of at
// most `suspend_ns` each.  Returns false when the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint32_t limit,
                                          uint32_t suspend_ns = MBAR_SUSPEND_NS)
{
    for (uint32_t i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity, suspend_ns)) return true;
    return false;
}

}  // namespace dvl

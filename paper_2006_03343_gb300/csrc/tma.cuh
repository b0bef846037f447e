// Inline-PTX helpers for the bulk-copy (TMA) pipelines: mbarrier set-up,
// arrive / expect-tx, bounded parity waits and 1D global->shared bulk copies.
#pragma once

#include <stdint.h>

namespace wmibm {

// Device status codes written by bounded waits that give up.
constexpr int kDevStatusOk = 0;
constexpr int kDevStatusFullTimeout = 1;    // a consumer waited too long for a stage's data
constexpr int kDevStatusEmptyTimeout = 2;   // the producer waited too long for a free stage
constexpr int kDevStatusBarrierTimeout = 3; // a block waited too long at the grid barrier

// A bounded wait gives up after this many nanoseconds of %globaltimer, or as
// soon as another wait of the same handle has given up (status != 0).
constexpr uint64_t kWaitLimitNs = 1000000000ull;

// Suspend-time hint of a try_wait: the waiting thread sleeps until the phase
// completes or this many nanoseconds pass, instead of spinning.
constexpr uint32_t kSuspendHintNs = 20000;

__device__ __forceinline__ uint64_t global_timer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(kSuspendHintNs)
        : "memory");
    return ok != 0;
}

// Waits for the phase of `bar` with the given parity to complete.  Gives up
// (returns false) after limit_ns of %globaltimer, recording `code` in *status,
// or at once if *status already holds a code.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *status, int code,
                                          uint64_t limit_ns = kWaitLimitNs)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 7u) == 0) {
            if (*(volatile int *)status != 0) return false;
            if (global_timer_ns() - t0 > limit_ns) {
                atomicExch(status, code);
                return false;
            }
        }
    }
}

// Waits (bounded by kWaitLimitNs, whatever the status word says) for the phase
// of `bar` with the given parity: used before a block that gave up exits, so
// that no bulk copy it issued still lands in its shared memory afterwards.
__device__ __forceinline__ void mbar_drain(uint64_t *bar, uint32_t parity)
{
    const uint64_t t0 = global_timer_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_timer_ns() - t0 > kWaitLimitNs) return;
}

// 1D bulk copy global -> shared, completing `bytes` transaction bytes on `bar`.
// dst and src must be 16-byte aligned and bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

}  // namespace wmibm

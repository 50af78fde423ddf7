// mg_bulk.cuh -- 1-D bulk asynchronous copies from global to shared memory,
// completed on an mbarrier, with a bounded wait (PTX ISA: cp.async.bulk,
// mbarrier).  Used to stage the small levels of the tail kernel: one thread
// issues every copy, the copies run on the SM's bulk-copy engine at once
// instead of a loop of dependent vector loads per array.
//
// Rules the callers keep: shared and global addresses 16-byte aligned, sizes
// a multiple of 16 bytes, the total per phase below 2^20 bytes (the mbarrier
// transaction count).
#pragma once

#include <cuda_runtime.h>

namespace gbmg {

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    // make the initialised barrier visible to the bulk-copy (async) proxy
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One arrival that also announces `bytes` of copies completing on the barrier.
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Wait for the barrier phase `parity` to complete; false if it did not within
// `limit` polls (each poll may suspend the thread for a short, bounded time).
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity, long long limit)
{
    for (long long it = 0; it < limit; it++) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// polls before a staging wait gives up (the copies take microseconds)
constexpr long long kBulkWaitPolls = 1ll << 20;

}  // namespace gbmg

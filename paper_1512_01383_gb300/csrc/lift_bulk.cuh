// Bulk (TMA) copies between global and shared memory and the mbarrier that
// tracks them, as inline PTX for sm_100-class GPUs: one elected thread moves a
// contiguous run of records per copy; the other threads wait on the barrier.
//
// Every wait here is bounded: after kMaxPolls polls the waiting thread gives up
// and the caller records an error (no spin without a limit).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lift {

// About 2^24 polls of try_wait; each poll suspends the thread for at most a
// few microseconds, so a copy that never lands ends the wait within seconds.
constexpr unsigned kMaxPolls = 1u << 24;

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
    // make the initialised barrier visible to the asynchronous (bulk copy) proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Arrive once on the barrier and announce `bytes` of bulk copies that complete on it.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("{\n\t.reg .b64 st;\n\t"
                 "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}"
                 ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Wait for phase `parity` of the barrier to complete; false if it did not
// within kMaxPolls polls.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity)
{
    const uint32_t a = smem_u32(bar);
    for (unsigned n = 0; n < kMaxPolls; ++n) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(a), "r"(parity)
                     : "memory");
        if (done) return true;
    }
    return false;
}

// Global -> shared, `bytes` (a multiple of 16) from a 16-byte aligned source
// to a 16-byte aligned destination, completing on `bar`.
__device__ __forceinline__ void bulk_load(void *dst_smem, const void *src, uint32_t bytes,
                                          uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
                 "[%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst_smem)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Shared -> global, same alignment rules; part of the thread's bulk group.
__device__ __forceinline__ void bulk_store(void *dst, const void *src_smem, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;"
                 ::"l"(dst), "r"(smem_u32(src_smem)), "r"(bytes)
                 : "memory");
}

// Prefetch `bytes` (a multiple of 16) from a 16-byte aligned global address
// into L2, with no destination and no completion to wait for.
__device__ __forceinline__ void bulk_prefetch_l2(const void *src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// Order this thread's earlier generic-proxy writes to shared memory (made
// visible to it by a block barrier) before later bulk copies read it.
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Close the thread's current group of bulk stores.
__device__ __forceinline__ void bulk_store_commit()
{
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// Wait until every committed bulk store of the thread has read its shared
// memory (the source may then be overwritten).
__device__ __forceinline__ void bulk_wait_read()
{
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// Wait until every committed bulk store of the thread has completed.
__device__ __forceinline__ void bulk_wait_all()
{
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

}  // namespace lift

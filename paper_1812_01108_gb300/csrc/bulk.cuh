// Bulk copies between global and shared memory through the TMA engine
// (cp.async.bulk, not tensor-mapped), shared by the chain kernels.
#pragma once

#include <stdint.h>

#include "sched.cuh"
#include "tpl_common.cuh"

namespace tpl {

// Bulk copies through the TMA engine (cp.async.bulk, not tensor-mapped): one
// thread moves a 16-byte aligned run of global memory into this CTA's shared
// memory, and an mbarrier counts the bytes in.  Every wait is bounded.
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// Orders this thread's generic shared-memory accesses before later
// async-proxy (bulk copy) accesses to the same memory.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One thread: the barrier's next phase expects `bytes`, and the copy delivers
// them.  The fence orders this CTA's earlier generic accesses to the stage
// before the async-proxy writes.
__device__ __forceinline__ void bulk_load(float* dst, const float* src, unsigned bytes, uint64_t* bar) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// Two bulk copies counted by one barrier phase: one arrival that expects the
// bytes of both.
__device__ __forceinline__ void bulk_load2(float* dst1, const float* src1, float* dst2, const float* src2,
                                           unsigned bytes, uint64_t* bar) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(2u * bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(dst1)), "l"(src1), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(dst2)), "l"(src2), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, unsigned phase) {
    unsigned done;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(done)
                 : "r"(smem_addr(bar)), "r"(phase)
                 : "memory");
    return done != 0;
}

// Bounded wait for the phase to complete; a give-up sets TPL_STATUS_TIMEOUT
// and then waits once more (bounded) so that no copy lands after the CTA has
// moved on if it can be helped.
__device__ __forceinline__ void mbar_wait(uint64_t* bar, unsigned phase) {
    for (int round = 0; round < 2; ++round) {
        for (int it = 0; it < kSpinLimit; ++it) {
            if (mbar_test(bar, phase)) return;
            if (it >= kSpinFast) __nanosleep(100);
        }
        if (round == 0 && threadIdx.x == 0) flag_status(TPL_STATUS_TIMEOUT);
    }
}

// Bulk store (TMA engine) of a 16-byte aligned run of this CTA's shared
// memory to global memory, issued by one thread into a bulk group.  Before the
// run is overwritten the thread waits for the group's reads
// (bulk_store_wait_read); before the kernel ends, for its writes.
__device__ __forceinline__ void bulk_store(float* dst, const float* src, unsigned bytes) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src)),
                 "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_store_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_store_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

}  // namespace tpl

// tma.cuh -- bulk asynchronous copies (the TMA engine) from global into shared memory, completed
// on a shared-memory transaction barrier (mbarrier), in inline PTX for sm_100-class GPUs.
//
// One thread initialises the barrier for one arrival, announces the bytes the copies will deliver
// (arrive + expect_tx) and issues the copies; every thread then polls the barrier's phase with a
// bounded number of tries, so that a copy that never lands ends in an error flag, not a hang.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ddrw {

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t arrivals)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(arrivals) : "memory");
}

// makes the initialised barrier visible to the copy engine
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// this thread's arrival, announcing `bytes` of copies that complete on the barrier
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

// bytes (a multiple of 16, both addresses 16-byte aligned) from global to this CTA's shared memory
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Polls the barrier until the phase of the given parity has completed, at most `tries` times with
// a short sleep in between (the copies are tracked by the barrier: when it completes they have
// landed).  Returns false when the tries run out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int tries)
{
    for (int i = 0; i < tries; i++) {
        if (mbar_test(bar, parity)) return true;
        __nanosleep(64);
    }
    return false;
}

}  // namespace ddrw

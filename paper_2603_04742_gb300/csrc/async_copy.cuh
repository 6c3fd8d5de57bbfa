// Bulk asynchronous copies (the TMA engine's cp.async.bulk) into shared
// memory, completed on an mbarrier, and bounded waits on them.
//
// Every wait gives up after a fixed number of polls: it then records
// kErrWaitTimeout in the context's device error word and returns false, and
// the kernel skips the rest of its work; hespmv_device_status reports it as
// HESPMV_E_TIMEOUT.  No wait can hang the GPU.
#pragma once
#include <cstdint>

namespace hespmv {

constexpr int kErrWaitTimeout = 1;
constexpr uint32_t kWaitPolls = 1u << 20;

#ifdef __CUDACC__
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// make the initialised barriers visible to the async proxy
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// order this thread's earlier generic-proxy accesses of shared memory before
// later async-proxy writes to it (a buffer about to be refilled)
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// one thread: expect `bytes` on `bar` and start the copy global -> shared
// (both 16-byte aligned, bytes a multiple of 16)
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// wait for phase `parity` of `bar` to complete, at most `polls` polls
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t polls, int *err) {
    const uint32_t a = smem_u32(bar);
    for (uint32_t it = 0; it < polls; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    if (err) atomicExch(err, kErrWaitTimeout);
    return false;
}
#endif

}  // namespace hespmv

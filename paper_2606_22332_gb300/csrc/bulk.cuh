// bulk.cuh -- bulk copies from HBM into shared memory (cp.async.bulk,
// completed on an mbarrier with a byte count) and the bounded mbarrier wait
// of the pipelined step kernel.
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

namespace tg {

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(saddr(dst)), "l"(src), "r"(bytes), "r"(saddr(mbar)) : "memory");
}

// an mbarrier with one expected arrival per phase
__device__ __forceinline__ void mbar_init(uint64_t* mbar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(saddr(mbar)));
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// the barrier's phase completes once `bytes` have landed (the arrival is this thread's)
__device__ __forceinline__ void mbar_expect(uint64_t* mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(saddr(mbar)), "r"(bytes) : "memory");
}

// bounded wait for the phase of the given parity; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity) {
    const uint32_t a = saddr(mbar);
    uint32_t done = 0;
    for (int it = 0; it < (1 << 22) && !done; ++it)
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
    return done != 0;
}

// orders this CTA's generic-proxy accesses of shared memory before the
// bulk copies issued after it
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Bulk copy of n elements of esz bytes starting at element `first` of
// `base`, from the 16-byte boundary at or below it to the one at or above
// its end (the buffers in HBM carry at least 16 bytes of slack past their
// end).  Adds the bytes to tx; returns the lead-in in elements.
__device__ __forceinline__ int stage(void* dst, const void* base, int64_t first, int n, int esz, uint64_t* mbar,
                                     uint32_t& tx) {
    const uintptr_t a = (uintptr_t)base + (uintptr_t)first * (uintptr_t)esz;
    const uintptr_t a0 = a & ~(uintptr_t)15;
    const uintptr_t a1 = (a + (uintptr_t)n * (uintptr_t)esz + 15) & ~(uintptr_t)15;
    const uint32_t bytes = (uint32_t)(a1 - a0);
    if (bytes) bulk_load(dst, reinterpret_cast<const void*>(a0), bytes, mbar);
    tx += bytes;
    return (int)((a - a0) / (uintptr_t)esz);
}

// 32-byte record from global memory into shared memory by cp.async (the
// issuing thread waits for it with cp_async_wait)
__device__ __forceinline__ void cp_async32(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(saddr(dst)), "l"(src) : "memory");
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(saddr(static_cast<char*>(dst) + 16)),
                 "l"(static_cast<const char*>(src) + 16) : "memory");
    asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

}  // namespace tg

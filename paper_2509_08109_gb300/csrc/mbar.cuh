// mbar.cuh -- shared-memory mbarrier and bulk-copy primitives (inline PTX)
// used by the kernels that stage data with the asynchronous copy engine.
// Every wait is bounded by the global timer so that a copy that never
// completes turns into an error status instead of a hung kernel.
#pragma once

#include <cuda.h>
#include <stdint.h>

namespace bmg {
namespace mbar {

constexpr unsigned long long kWaitNs = 2000000000ull;   // 2 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void init(uint64_t* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool try_wait(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for phase `parity` of the barrier; false once kWaitNs have passed.
__device__ __forceinline__ bool wait(uint64_t* b, uint32_t parity) {
    if (try_wait(b, parity)) return true;
    const unsigned long long t0 = gtimer();
    while (!try_wait(b, parity))
        if (gtimer() - t0 > kWaitNs) return false;
    return true;
}

// Untiled bulk copy global -> this CTA's shared memory, completing `bytes`
// on the barrier.  Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"((unsigned long long)src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

}  // namespace mbar
}  // namespace bmg

// Bulk asynchronous copies (cp.async.bulk, the TMA engine's untiled form) completing on shared
// memory barriers, for kernels that stream tiles through shared memory.
//
// Waits are bounded: mbar_wait gives up after `limit` polls (each poll may suspend the thread for
// a short, system-defined time), so a copy that never completes makes the kernel report
// LC_ERR_TIMEOUT through the context's error word instead of spinning forever.
#pragma once
#include <cstdint>

// bits of the context's device error word (reported by lc_sync)
#define LC_ERR_TIMEOUT 1u   // a bounded wait on a shared-memory barrier gave up
#define LC_ERR_RANGE 2u     // a wire-form residue was not below its prime
constexpr unsigned kMbarPolls = 1u << 22;

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// makes barrier initialisation visible to the asynchronous proxy (the copy engine)
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// orders this thread's earlier generic-proxy shared-memory accesses before later bulk copies
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// the calling thread arrives and announces `bytes` of transfer for the current phase
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// global -> shared copy of `bytes` (multiple of 16, both addresses 16-byte aligned), completing
// as transaction bytes on `bar`
__device__ __forceinline__ void bulk_load(void* dst_smem, const void* src_gmem, unsigned bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// waits for phase `parity` of `bar` to complete; false if it did not within the poll limit
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, unsigned limit = kMbarPolls) {
    for (unsigned it = 0; it < limit; it++) {
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

// Integer-pipe probes: register-resident kernels that measure how fast this GPU retires the
// 32-bit integer multiply-adds from which every 64-bit modular product here is built.  They touch
// no memory except one conditional word at exit (so the compiler keeps the arithmetic), and serve
// only as the measured ceiling beside which the arithmetic-bound kernels are reported.
#include <cuda_runtime.h>
#include <cstdint>
#include "probe.cuh"
#include "tma.cuh"

namespace {

constexpr int kChains = 8;  // independent dependency chains per thread

// x_k <- x_k*m + x_{k+1} on 32-bit words (mad.lo.u32; the coupling keeps the compiler from
// folding a chain into a closed form); c only seeds the chains
__global__ void __launch_bounds__(kProbeThreads) k_probe_imad(uint32_t m, uint32_t c, uint32_t iters,
                                                              unsigned long long* sink) {
    uint32_t x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) x[k] = threadIdx.x + 977u * k + blockIdx.x + c;
    for (uint32_t it = 0; it < iters; it++) {
#pragma unroll
        for (int r = 0; r < 8; r++) {
            uint32_t y[kChains];
#pragma unroll
            for (int k = 0; k < kChains; k++) y[k] = x[k] * m + x[(k + 1) % kChains];
#pragma unroll
            for (int k = 0; k < kChains; k++) x[k] = y[k];
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int k = 0; k < kChains; k++) acc ^= x[k];
    if (acc == 0x9e3779b9u) atomicAdd(sink, 1ull);
}

// x_k <- lo32(x_k) * m + x_{k+1} as a 32x32 -> 64-bit multiply-add (mad.wide.u32)
__global__ void __launch_bounds__(kProbeThreads) k_probe_imad_wide(uint32_t m, uint32_t iters,
                                                                   unsigned long long* sink) {
    uint64_t x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) x[k] = threadIdx.x + 977ull * k + blockIdx.x;
    for (uint32_t it = 0; it < iters; it++) {
#pragma unroll
        for (int r = 0; r < 8; r++) {
            uint64_t y[kChains];
#pragma unroll
            for (int k = 0; k < kChains; k++) y[k] = (uint64_t)(uint32_t)x[k] * m + x[(k + 1) % kChains];
#pragma unroll
            for (int k = 0; k < kChains; k++) x[k] = y[k];
        }
    }
    uint64_t acc = 0;
#pragma unroll
    for (int k = 0; k < kChains; k++) acc ^= x[k];
    if (acc == 0x9e3779b97f4a7c15ull) atomicAdd(sink, 1ull);
}

// Self-test of the bounded shared-memory-barrier wait used by the bulk-copy kernels.  One block
// of 32 threads: thread 0 streams 64 bytes into shared memory with a bulk copy completing on
// barrier A, and all threads wait on A (bounded); the copy is then written back to `dst`.  With
// `never_arrive`, the block afterwards waits on a barrier B at which nothing ever arrives, so the
// wait runs out after `max_polls` polls and the block reports LC_ERR_TIMEOUT in `err`; no copy is
// in flight at that point (A completed first).
__global__ void __launch_bounds__(32) k_wait_selftest(const unsigned long long* __restrict__ src,
                                                      unsigned long long* __restrict__ dst, int never_arrive,
                                                      unsigned max_polls, unsigned* err) {
    __shared__ __align__(128) unsigned long long buf[8];
    __shared__ __align__(8) uint64_t bar[2];
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(&bar[0], sizeof(buf));
        bulk_load(buf, src, sizeof(buf), &bar[0]);
    }
    if (!__syncthreads_and(mbar_wait(&bar[0], 0, max_polls))) {
        if (threadIdx.x == 0) atomicOr(err, LC_ERR_TIMEOUT);
        return;
    }
    if (threadIdx.x < 8) dst[threadIdx.x] = buf[threadIdx.x];
    if (never_arrive && !__syncthreads_and(mbar_wait(&bar[1], 0, max_polls)) && threadIdx.x == 0)
        atomicOr(err, LC_ERR_TIMEOUT);
}

}  // namespace

void wait_selftest(const unsigned long long* src, unsigned long long* dst, int never_arrive, unsigned max_polls,
                   unsigned* err, cudaStream_t s) {
    k_wait_selftest<<<1, 32, 0, s>>>(src, dst, never_arrive, max_polls, err);
}

void probe_imad(int blocks, uint32_t iters, unsigned long long* sink, cudaStream_t s) {
    k_probe_imad<<<blocks, kProbeThreads, 0, s>>>(0x2545f491u, 0x9e3779b9u ^ 1u, iters, sink);
}
void probe_imad_wide(int blocks, uint32_t iters, unsigned long long* sink, cudaStream_t s) {
    k_probe_imad_wide<<<blocks, kProbeThreads, 0, s>>>(0x2545f491u, iters, sink);
}

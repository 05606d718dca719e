// Integer-pipe probes: register-resident kernels that measure how fast this GPU retires the
// 32-bit integer multiply-adds from which every 64-bit modular product here is built.  They touch
// no memory except one conditional word at exit (so the compiler keeps the arithmetic), and serve
// only as the measured ceiling beside which the arithmetic-bound kernels are reported.
#include <cuda_runtime.h>
#include <cstdint>
#include "probe.cuh"

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

}  // namespace

void probe_imad(int blocks, uint32_t iters, unsigned long long* sink, cudaStream_t s) {
    k_probe_imad<<<blocks, kProbeThreads, 0, s>>>(0x2545f491u, 0x9e3779b9u ^ 1u, iters, sink);
}
void probe_imad_wide(int blocks, uint32_t iters, unsigned long long* sink, cudaStream_t s) {
    k_probe_imad_wide<<<blocks, kProbeThreads, 0, s>>>(0x2545f491u, iters, sink);
}

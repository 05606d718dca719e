// Launchers of the integer-pipe probe kernels (probe.cu; the butterfly probe lives in ntt.cu
// beside the butterfly it measures).  Each thread executes `iters` x 64 operations (8 chains x 8
// unrolled steps per iteration; the butterfly probe: 32 butterflies per iteration).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

constexpr int kProbeThreads = 256;

void probe_imad(int blocks, uint32_t iters, unsigned long long* sink, cudaStream_t s);
void probe_imad_wide(int blocks, uint32_t iters, unsigned long long* sink, cudaStream_t s);
void probe_ntt_bfly(int blocks, uint32_t iters, unsigned long long* sink, cudaStream_t s);
// bounded-wait self-test (probe.cu): src/dst are 64-byte device buffers (16-byte aligned)
void wait_selftest(const unsigned long long* src, unsigned long long* dst, int never_arrive, unsigned max_polls,
                   unsigned* err, cudaStream_t s);

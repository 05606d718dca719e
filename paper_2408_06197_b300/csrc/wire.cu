// Wire form of ciphertext arrays: every residue of limb i (canonical, below q_i) is stored in
// w_i = ceil(bits(q_i - 1) / 8) little-endian bytes instead of a 64-bit word, limb after limb,
// so a production ciphertext at level 14 (one 60-bit and fourteen 40-bit primes) moves 78 bytes
// per coefficient instead of 120.  Each thread converts a group of 16 residues: 16 w_i bytes =
// w_i aligned 16-byte vectors on the wire side, 128 bytes on the word side, so both sides are
// read and written in whole 16-byte vectors by consecutive threads.
#include <cuda_runtime.h>
#include <cstdint>
#include "wire.cuh"
#include "tma.cuh"

namespace {

constexpr int kWT = 256;

// bits [8 W k, 8 W k + 8 W) of the little-endian word array wd (compile-time positions)
template <int W>
__device__ __forceinline__ uint64_t take(const uint32_t* wd, int k) {
    const int bit = 8 * W * k, wi = bit >> 5, sh = bit & 31;
    uint64_t v = (uint64_t)wd[wi] >> sh;
    if (wi + 1 < 4 * W) v |= (uint64_t)wd[wi + 1] << (32 - sh);
    if (sh && wi + 2 < 4 * W && 8 * W + sh > 64) v |= (uint64_t)wd[wi + 2] << (64 - sh);
    return W == 8 ? v : v & ((1ull << (8 * W)) - 1);
}

template <int W>
__device__ __forceinline__ void put(uint32_t* wd, int k, uint64_t v) {
    const int bit = 8 * W * k, wi = bit >> 5, sh = bit & 31;
    wd[wi] |= (uint32_t)(v << sh);
    if (wi + 1 < 4 * W) wd[wi + 1] |= (uint32_t)(v >> (32 - sh));
    if (sh && wi + 2 < 4 * W && 8 * W + sh > 64) wd[wi + 2] |= (uint32_t)(v >> (64 - sh));
}

template <int W>
__device__ __forceinline__ void unpack16(const uint4* src, uint64_t* dst, uint64_t q, unsigned* err) {
    uint32_t wd[4 * W];
#pragma unroll
    for (int i = 0; i < W; i++) {
        const uint4 v = __ldg(src + i);
        wd[4 * i] = v.x;
        wd[4 * i + 1] = v.y;
        wd[4 * i + 2] = v.z;
        wd[4 * i + 3] = v.w;
    }
    bool bad = false;
#pragma unroll
    for (int k = 0; k < 16; k += 2) {
        const uint64_t a = take<W>(wd, k), b = take<W>(wd, k + 1);
        bad |= a >= q || b >= q;
        *reinterpret_cast<ulonglong2*>(dst + k) = make_ulonglong2(a, b);
    }
    if (bad) atomicOr(err, LC_ERR_RANGE);
}

template <int W>
__device__ __forceinline__ void pack16(const uint64_t* src, uint4* dst) {
    uint32_t wd[4 * W];
#pragma unroll
    for (int i = 0; i < 4 * W; i++) wd[i] = 0;
#pragma unroll
    for (int k = 0; k < 16; k += 2) {
        const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(src + k);
        put<W>(wd, k, v.x);
        put<W>(wd, k + 1, v.y);
    }
#pragma unroll
    for (int i = 0; i < W; i++) dst[i] = make_uint4(wd[4 * i], wd[4 * i + 1], wd[4 * i + 2], wd[4 * i + 3]);
}

// unit u = ((record * deg + poly) * nl + limb) * (N / 16) + group
__global__ void __launch_bounds__(kWT) k_unpack(const unsigned char* __restrict__ in, uint64_t* __restrict__ out,
                                                size_t units, WireMap m, unsigned* err) {
    const size_t G = (size_t)1 << (m.log_n - 4);
    for (size_t u = (size_t)blockIdx.x * blockDim.x + threadIdx.x; u < units; u += (size_t)gridDim.x * blockDim.x) {
        const size_t g = u & (G - 1), rest = u >> (m.log_n - 4);
        const int i = (int)(rest % m.nl);
        const size_t rp = rest / m.nl;
        const int w = m.w[i];
        const uint4* src = reinterpret_cast<const uint4*>(in + rp * m.poly_bytes + m.off[i] + g * 16 * (size_t)w);
        uint64_t* dst = out + (rp * m.nl + i) * (G << 4) + g * 16;
        const uint64_t q = m.q[i];
        switch (w) {
            case 4: unpack16<4>(src, dst, q, err); break;
            case 5: unpack16<5>(src, dst, q, err); break;
            case 6: unpack16<6>(src, dst, q, err); break;
            case 7: unpack16<7>(src, dst, q, err); break;
            default: unpack16<8>(src, dst, q, err); break;
        }
    }
}

__global__ void __launch_bounds__(kWT) k_pack(const uint64_t* __restrict__ in, unsigned char* __restrict__ out,
                                              size_t units, WireMap m) {
    const size_t G = (size_t)1 << (m.log_n - 4);
    for (size_t u = (size_t)blockIdx.x * blockDim.x + threadIdx.x; u < units; u += (size_t)gridDim.x * blockDim.x) {
        const size_t g = u & (G - 1), rest = u >> (m.log_n - 4);
        const int i = (int)(rest % m.nl);
        const size_t rp = rest / m.nl;
        const int w = m.w[i];
        uint4* dst = reinterpret_cast<uint4*>(out + rp * m.poly_bytes + m.off[i] + g * 16 * (size_t)w);
        const uint64_t* src = in + (rp * m.nl + i) * (G << 4) + g * 16;
        switch (w) {
            case 4: pack16<4>(src, dst); break;
            case 5: pack16<5>(src, dst); break;
            case 6: pack16<6>(src, dst); break;
            case 7: pack16<7>(src, dst); break;
            default: pack16<8>(src, dst); break;
        }
    }
}

unsigned wire_grid(size_t units) {
    const size_t b = (units + kWT - 1) / kWT;
    return (unsigned)(b < 148 * 16 ? (b ? b : 1) : 148 * 16);
}

}  // namespace

void wire_unpack(const unsigned char* in, uint64_t* out, size_t polys, const WireMap& m, unsigned* err,
                 cudaStream_t s) {
    const size_t units = polys * m.nl * ((size_t)1 << (m.log_n - 4));
    if (units) k_unpack<<<wire_grid(units), kWT, 0, s>>>(in, out, units, m, err);
}

void wire_pack(const uint64_t* in, unsigned char* out, size_t polys, const WireMap& m, cudaStream_t s) {
    const size_t units = polys * m.nl * ((size_t)1 << (m.log_n - 4));
    if (units) k_pack<<<wire_grid(units), kWT, 0, s>>>(in, out, units, m);
}

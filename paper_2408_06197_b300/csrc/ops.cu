// Evaluation kernels of the Lancelot server path (elementwise RNS arithmetic, tensor and
// lazy accumulation, base conversion, key inner product, rescale, automorphism).
#include <cuda_runtime.h>
#include <mutex>
#include <set>
#include <algorithm>
#include "ops.cuh"

std::atomic<uint64_t> g_lc_launches{0};

namespace {

constexpr int kT = 256;  // threads per block for elementwise kernels

struct ModList {
    int n;
    uint8_t m[LC_MAX_ROWS];
    uint8_t flag[LC_MAX_ROWS];
    u64 val[LC_MAX_ROWS];
};

// up to 15 rotations of one hoisted group (groups of at most 4 rotation bits)
struct KeyPtrs {
    const u64* p[16];
};
struct Galois {
    uint64_t g[16];
};

ModList make_list(const int* mods, int n, const u64* vals = nullptr) {
    ModList l{};
    l.n = n;
    for (int i = 0; i < n && i < LC_MAX_ROWS; i++) {
        l.m[i] = (uint8_t)mods[i];
        l.val[i] = vals ? vals[i] : 0;
        l.flag[i] = vals ? (vals[i] != 0) : 0;
    }
    return l;
}

__device__ __forceinline__ u64 reduce64(u64 v, const ModConst& m) {
    return csub(v - __umul64hi(v, m.one_sh) * m.q, m.q);
}

__device__ __forceinline__ u64 signed_to_res(int64_t v, const ModConst& m) {
    u64 a = v < 0 ? (u64)(-(v + 1)) + 1 : (u64)v;  // |v| without overflow
    u64 r = reduce64(a, m);
    return (v < 0 && r) ? m.q - r : r;
}

// perm_g(idx): the source index of the automorphism X -> X^g in the bit-reversed evaluation
// order: out[idx] = in[perm_g(idx)], with 2 br(src)+1 = g (2 br(idx)+1) mod 2N.
__device__ __forceinline__ unsigned auto_src(unsigned idx, uint64_t g, int log_n) {
    const unsigned k = __brev(idx) >> (32 - log_n);
    const uint64_t e = (g * (2ull * k + 1)) & ((2ull << log_n) - 1);
    const unsigned k2 = (unsigned)((e - 1) >> 1);
    return __brev(k2) >> (32 - log_n);
}

// ---------------------------------------------------------------------------- elementwise
__global__ void k_addsub(const u64* __restrict__ a, const u64* __restrict__ b, u64* __restrict__ out, int nl,
                         int log_n, size_t total, const ModConst* __restrict__ mc, int sub) {
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
        const int limb = (int)((idx >> log_n) % nl);
        const u64 q = mc[limb].q;
        out[idx] = sub ? sub_mod(a[idx], b[idx], q) : add_mod(a[idx], b[idx], q);
    }
}

__global__ void k_tensor(const u64* __restrict__ a, const u64* __restrict__ b, u64* __restrict__ out, int log_n,
                         size_t P, const ModConst* __restrict__ mc) {
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < P; idx += (size_t)gridDim.x * blockDim.x) {
        const ModConst m = mc[idx >> log_n];
        const u64 a0 = a[idx], a1 = a[P + idx], b0 = b[idx], b1 = b[P + idx];
        u128v s0{0, 0}, s1{0, 0}, s2{0, 0};
        mac128(s0, a0, b0);
        mac128(s1, a0, b1);
        mac128(s1, a1, b0);
        mac128(s2, a1, b1);
        out[idx] = reduce128(s0, m);
        out[P + idx] = reduce128(s1, m);
        out[2 * P + idx] = reduce128(s2, m);
    }
}

// (i, j) of pair p in lexicographic i<j order
__device__ __forceinline__ void pair_of(int p, int n, int& i, int& j) {
    i = 0;
    while (p >= n - 1 - i) {
        p -= n - 1 - i;
        i++;
    }
    j = i + 1 + p;
}

__device__ __forceinline__ void fold(u128v& s, const ModConst& m) {
    s.lo = reduce128(s, m);
    s.hi = 0;
}

// grid: x = pair (fastest, so all pairs of one coefficient tile run together and share the
// clients' tiles through L2), y = coefficient tile, z = limb
__global__ void __launch_bounds__(kT) k_sq_acc_pairs(const u64* __restrict__ cts, int n, int chunks, int nl, int log_n,
                                                     int p0, const ModConst* __restrict__ mc, u64* __restrict__ out) {
    const int p = p0 + blockIdx.x;
    const int limb = blockIdx.z;
    const size_t x = (size_t)blockIdx.y * kT + threadIdx.x;
    const size_t N = (size_t)1 << log_n;
    int i, j;
    pair_of(p, n, i, j);
    const ModConst m = mc[limb];
    const size_t P = (size_t)nl * N;
    const u64* ai = cts + (size_t)i * chunks * 2 * P + (size_t)limb * N + x;
    const u64* aj = cts + (size_t)j * chunks * 2 * P + (size_t)limb * N + x;
    u128v s00{0, 0}, s01{0, 0}, s11{0, 0};
    for (int k = 0; k < chunks; k++) {
        const u64 a0 = __ldg(ai), a1 = __ldg(ai + P), b0 = __ldg(aj), b1 = __ldg(aj + P);
        ai += 2 * P;
        aj += 2 * P;
        const u64 x0 = sub_mod(a0, b0, m.q), x1 = sub_mod(a1, b1, m.q);
        mac128(s00, x0, x0);
        mac128(s01, x0, x1);
        mac128(s11, x1, x1);
        if ((k & 7) == 7) {
            fold(s00, m);
            fold(s01, m);
            fold(s11, m);
        }
    }
    u64* o = out + (size_t)blockIdx.x * 3 * P + (size_t)limb * N + x;
    o[0] = reduce128(s00, m);
    const u64 d1 = reduce128(s01, m);
    o[P] = add_mod(d1, d1, m.q);
    o[2 * P] = reduce128(s11, m);
}

// Batched distances tensor phase with client-block tiling.  Clients are grouped in blocks of
// `cb` (all clients when n <= 11, else 8); a CTA owns one pair of client blocks (I <= J), one
// 32-coefficient tile and one limb.  Chunk tiles of all its clients stream through a
// shared-memory ring of kRing stages of kCPS chunks, filled with cp.async (kRing - 1 stages in
// flight, one block barrier per stage); each warp owns a set of pairs and one lane per
// coefficient, and accumulates (a-b)^2 for every chunk.
// Each client tile is read from HBM about n/cb times instead of n-1 times.  Pairs outside
// [p0, p0+np) are skipped (waves).
constexpr int kTX = 32;
#ifndef LC_TENSOR_RING
#define LC_TENSOR_RING 3
#endif
#ifndef LC_TENSOR_CPS
#define LC_TENSOR_CPS 4
#endif
constexpr int kMaxSlots = 16;                  // client slots staged per chunk (2 blocks of 8, or 11)
constexpr int kRing = LC_TENSOR_RING;  // ring stages (kRing - 1 groups in flight)
constexpr int kCPS = LC_TENSOR_CPS;    // chunks per stage (one barrier per stage)
constexpr size_t kTensorSmem = (size_t)kRing * kCPS * kMaxSlots * 2 * kTX * 8;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N_>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N_)); }

// Exact sums of products of residues below 2^40 without 128-bit carry chains: each operand is
// split into 20-bit halves (v = h 2^20 + l), each partial product is one 32x32 -> 64-bit
// multiply-add, and the three weights (2^40, 2^20, 1) accumulate separately in 64 bits (each
// term < 2^41, so up to 2^20 chunks cannot overflow).
struct Acc3 {
    u64 a, b, c;  // sum h h', sum (h l' + l h'), sum l l'
};
__device__ __forceinline__ void mac_split(Acc3& s, unsigned h, unsigned l, unsigned h2, unsigned l2) {
    s.a += (u64)h * h2;
    s.b += (u64)h * l2;
    s.b += (u64)l * h2;
    s.c += (u64)l * l2;
}
// Karatsuba form: b collects (h + l)(h2 + l2); the caller subtracts a + c once at the end
__device__ __forceinline__ void mac_kara(Acc3& s, unsigned h, unsigned l, unsigned hl, unsigned h2, unsigned l2) {
    s.a += (u64)h * h2;
    s.b += (u64)hl * (h2 + l2);
    s.c += (u64)l * l2;
}
// the same as explicit 32-bit multiply-adds with a carry chain into the two halves of each
// 64-bit partial sum (measured faster than 64-bit wide multiply-adds in the distance tensor
// kernel, slower in the others)
__device__ __forceinline__ void mad_wide(u64& acc, unsigned a, unsigned b) {
    unsigned lo = (unsigned)acc, hi = (unsigned)(acc >> 32);
    asm("mad.lo.cc.u32 %0, %2, %3, %0;\n\tmadc.hi.u32 %1, %2, %3, %1;" : "+r"(lo), "+r"(hi) : "r"(a), "r"(b));
    acc = ((u64)hi << 32) | lo;
}
__device__ __forceinline__ void mac_split_w(Acc3& s, unsigned h, unsigned l, unsigned h2, unsigned l2) {
    mad_wide(s.a, h, h2);
    mad_wide(s.b, h, l2);
    mad_wide(s.b, l, h2);
    mad_wide(s.c, l, l2);
}
__device__ __forceinline__ void sq_split_w(Acc3& s, unsigned h, unsigned l) {  // b holds sum h l (doubled later)
    mad_wide(s.a, h, h);
    mad_wide(s.b, h, l);
    mad_wide(s.c, l, l);
}
// a 2^40 + b 2^20 * bmul + c mod q
__device__ __forceinline__ u64 acc3_reduce(const Acc3& s, int bshift, const ModConst& m) {
    u128v v{s.c, 0};
    add128(v, s.a << 40);
    v.hi += s.a >> 24;
    add128(v, s.b << bshift);
    v.hi += s.b >> (64 - bshift);
    return reduce128(v, m);
}

// WARPS warps, PPT pair slots per thread; SPLIT: the limbs' primes are below 2^40 (20-bit split
// arithmetic), else 128-bit multiply-accumulate with a fold every 8 chunks.  Limb = limb0 + z.
template <int WARPS, int PPT, bool SPLIT>
__global__ void __launch_bounds__(WARPS * 32, (SPLIT || WARPS > 8) ? 1 : 2) k_sq_acc_tiled(const u64* __restrict__ cts, int n, int chunks,
                                                                int nl, int limb0, int log_n, int cb, int p0, int np,
                                                                const ModConst* __restrict__ mc,
                                                                u64* __restrict__ out) {
    constexpr int NT = WARPS * 32;
    constexpr int UPT = (kMaxSlots * 2 * (kTX / 2) + NT - 1) / NT;  // 16-byte copy units per thread
    static_assert(WARPS * PPT >= 64, "pair slots must cover a block pair (8 x 8, or 55 pairs of 11 clients)");
    // ring of kRing stages of kCPS chunks each, in dynamic shared memory
    extern __shared__ __align__(16) u64 dyn_sh[];
    auto sh = reinterpret_cast<u64(*)[kMaxSlots][2][kTX]>(dyn_sh);
    constexpr int RS = kRing, CPS = kCPS;
    const int nb = (n + cb - 1) / cb;
    int bp = blockIdx.x, I = 0;
    while (bp >= nb - I) {
        bp -= nb - I;
        I++;
    }
    const int J = I + bp;
    const int cI0 = I * cb, cJ0 = J * cb;
    const int cntI = min(cb, n - cI0), cntJ = min(cb, n - cJ0);
    const bool diag = I == J;
    const int total = diag ? cntI * (cntI - 1) / 2 : cntI * cntJ;
    const int nslots = diag ? cntI : cntI + cntJ;
    const int limb = limb0 + blockIdx.z;
    const size_t N = (size_t)1 << log_n;
    const int tid = threadIdx.x, x = tid & 31, warp = tid >> 5;
    const size_t x0 = (size_t)blockIdx.y * kTX;
    const ModConst m = mc[limb];
    const size_t P = (size_t)nl * N;
    // per pair: (output index << 8) | (slot a << 4) | slot b, or -1 when the pair is not owned
    int pk[PPT];
    bool any = false;
#pragma unroll
    for (int k = 0; k < PPT; k++) {
        const int pi = warp + WARPS * k;
        pk[k] = -1;
        int sa = 0, sb = 0;
        if (pi < total) {
            int a, b;
            if (diag) {
                a = 0;
                int r = pi;
                while (r >= cntI - 1 - a) {
                    r -= cntI - 1 - a;
                    a++;
                }
                b = a + 1 + r;
                sa = a;
                sb = b;
            } else {
                a = pi / cntJ;
                b = pi - a * cntJ;
                sa = a;
                sb = cntI + b;
            }
            const int i = cI0 + a, j = (diag ? cI0 : cJ0) + b;
            const int g = i * n - i * (i + 1) / 2 + (j - i - 1);
            if (g >= p0 && g < p0 + np) {
                pk[k] = ((g - p0) << 8) | (sa << 4) | sb;
                any = true;
            }
        }
    }
    if (!__syncthreads_or(any)) return;
    // 16-byte copy units: (client slot, poly, coefficient pair): 32 per slot, <= 512 in all
    const int units = nslots * 2 * (kTX / 2);
    const u64* gsrc[UPT];
    int ucs[UPT], upp[UPT], uxx[UPT];
    bool ucopy[UPT];
#pragma unroll
    for (int h = 0; h < UPT; h++) {
        const int u = tid + h * NT;
        ucopy[h] = u < units;
        ucs[h] = u / kTX;
        upp[h] = (u / (kTX / 2)) & 1;
        uxx[h] = (u % (kTX / 2)) * 2;
        const int c = ucs[h] < cntI ? cI0 + ucs[h] : cJ0 + (ucs[h] - cntI);
        gsrc[h] = cts + ((size_t)(ucopy[h] ? c : 0) * chunks * 2 + upp[h]) * P + (size_t)limb * N + x0 + uxx[h];
    }
    const size_t chunk_stride = 2 * P;
    const int groups = (chunks + CPS - 1) / CPS;
#pragma unroll
    for (int st = 0; st < RS - 1; st++) {
#pragma unroll
        for (int c = 0; c < CPS; c++)
#pragma unroll
            for (int h = 0; h < UPT; h++)
                if (ucopy[h] && st * CPS + c < chunks)
                    cp_async16(&sh[st * CPS + c][ucs[h]][upp[h]][uxx[h]], gsrc[h] + (size_t)(st * CPS + c) * chunk_stride);
        cp_async_commit();
    }
    Acc3 t00[SPLIT ? PPT : 1], t01[SPLIT ? PPT : 1], t11[SPLIT ? PPT : 1];
    u128v s00[SPLIT ? 1 : PPT], s01[SPLIT ? 1 : PPT], s11[SPLIT ? 1 : PPT];
#pragma unroll
    for (int k = 0; k < PPT; k++) {
        if (SPLIT)
            t00[k] = t01[k] = t11[k] = Acc3{0, 0, 0};
        else
            s00[k] = s01[k] = s11[k] = u128v{0, 0};
    }
    // word offsets of each pair's two client slots inside one ring stage
    constexpr int STAGE = kMaxSlots * 2 * kTX;
    int oa[PPT], ob[PPT];
#pragma unroll
    for (int t = 0; t < PPT; t++) {
        oa[t] = ((pk[t] >> 4) & 15) * 2 * kTX + x;
        ob[t] = (pk[t] & 15) * 2 * kTX + x;
    }
    const u64* shf = &sh[0][0][0][0];
    const u64* pa[PPT];
    const u64* pb[PPT];
#pragma unroll
    for (int t = 0; t < PPT; t++) {
        pa[t] = shf + oa[t];
        pb[t] = shf + ob[t];
    }
    // one barrier per group of CPS chunks: the copies of group g + RS - 1 overlap groups g..;
    // the ring slot is a compile-time index (the loop over slots is unrolled), so every
    // shared-memory load is [pair base + constant]
    for (int g0 = 0; g0 < groups; g0 += RS) {
#pragma unroll
        for (int rs = 0; rs < RS; rs++) {
            const int gi = g0 + rs;
            if (gi >= groups) break;
            cp_async_wait<RS - 2>();
            __syncthreads();
            {
                const int ng = gi + RS - 1;
#pragma unroll
                for (int c = 0; c < CPS; c++)
#pragma unroll
                    for (int h = 0; h < UPT; h++)
                        if (ucopy[h] && ng * CPS + c < chunks)
                            cp_async16(&sh[((rs + RS - 1) % RS) * CPS + c][ucs[h]][upp[h]][uxx[h]],
                                       gsrc[h] + (size_t)(ng * CPS + c) * chunk_stride);
                cp_async_commit();
            }
#pragma unroll
            for (int c = 0; c < CPS; c++) {
                const int k = gi * CPS + c;
                if (k >= chunks) break;
                const int so = (rs * CPS + c) * STAGE;
#pragma unroll
                for (int t = 0; t < PPT; t++) {
                    if (pk[t] < 0) continue;
                    const u64 a0 = pa[t][so], a1 = pa[t][so + kTX];
                    const u64 b0 = pb[t][so], b1 = pb[t][so + kTX];
                    if (SPLIT) {
                        // a + q - b in [1, 2q): congruent to the difference, halves below 2^21, so
                        // every partial product stays below 2^42 and < 2^20 chunks cannot overflow
                        const u64 d0 = a0 + m.q - b0, d1 = a1 + m.q - b1;
                        const unsigned h0 = (unsigned)(d0 >> 20), l0 = (unsigned)d0 & 0xFFFFFu;
                        const unsigned h1 = (unsigned)(d1 >> 20), l1 = (unsigned)d1 & 0xFFFFFu;
                        sq_split_w(t00[t], h0, l0);
                        mac_split_w(t01[t], h0, l0, h1, l1);
                        sq_split_w(t11[t], h1, l1);
                    } else {
                        const u64 d0 = sub_mod(a0, b0, m.q), d1 = sub_mod(a1, b1, m.q);
                        mac128(s00[t], d0, d0);
                        mac128(s01[t], d0, d1);
                        mac128(s11[t], d1, d1);
                        if ((k & 7) == 7) {
                            fold(s00[t], m);
                            fold(s01[t], m);
                            fold(s11[t], m);
                        }
                    }
                }
            }
        }
    }
    cp_async_wait<0>();
#pragma unroll
    for (int t = 0; t < PPT; t++) {
        if (pk[t] < 0) continue;
        u64* o = out + (size_t)(pk[t] >> 8) * 3 * P + (size_t)limb * N + x0 + x;
        u64 r00, r01, r11;
        if (SPLIT) {
            r00 = acc3_reduce(t00[t], 21, m);
            r01 = acc3_reduce(t01[t], 20, m);
            r11 = acc3_reduce(t11[t], 21, m);
        } else {
            r00 = reduce128(s00[t], m);
            r01 = reduce128(s01[t], m);
            r11 = reduce128(s11[t], m);
        }
        o[0] = r00;
        o[P] = add_mod(r01, r01, m.q);
        o[2 * P] = r11;
    }
}

// grid: x = chunk (fastest; the masks are shared by every chunk), y = tile, z = limb
template <bool SPLIT>
__global__ void __launch_bounds__(kT) k_mask_acc(const u64* __restrict__ cts, int n, int chunks, int nl, int limb0,
                                                 int log_n, int k0, const u64* __restrict__ masks,
                                                 const ModConst* __restrict__ mc, u64* __restrict__ out) {
    const int k = k0 + blockIdx.x;
    const int limb = limb0 + blockIdx.z;
    const size_t x = (size_t)blockIdx.y * kT + threadIdx.x;
    const size_t N = (size_t)1 << log_n;
    const ModConst m = mc[limb];
    const size_t P = (size_t)nl * N;
    u128v s00{0, 0}, s01{0, 0}, s11{0, 0};
    Acc3 t00{0, 0, 0}, t01{0, 0, 0}, t11{0, 0, 0};
    for (int i = 0; i < n; i++) {
        const u64* a = cts + ((size_t)i * chunks + k) * 2 * P + (size_t)limb * N + x;
        const u64* w = masks + (size_t)i * 2 * P + (size_t)limb * N + x;
        const u64 a0 = __ldg(a), a1 = __ldg(a + P), m0 = __ldg(w), m1 = __ldg(w + P);
        if (SPLIT) {
            const unsigned ah0 = (unsigned)(a0 >> 20), al0 = (unsigned)a0 & 0xFFFFFu;
            const unsigned ah1 = (unsigned)(a1 >> 20), al1 = (unsigned)a1 & 0xFFFFFu;
            const unsigned mh0 = (unsigned)(m0 >> 20), ml0 = (unsigned)m0 & 0xFFFFFu;
            const unsigned mh1 = (unsigned)(m1 >> 20), ml1 = (unsigned)m1 & 0xFFFFFu;
            mac_split(t00, ah0, al0, mh0, ml0);
            mac_split(t01, ah0, al0, mh1, ml1);
            mac_split(t01, ah1, al1, mh0, ml0);
            mac_split(t11, ah1, al1, mh1, ml1);
        } else {
            mac128(s00, a0, m0);
            mac128(s01, a0, m1);
            mac128(s01, a1, m0);
            mac128(s11, a1, m1);
            if ((i & 3) == 3) {
                fold(s00, m);
                fold(s01, m);
                fold(s11, m);
            }
        }
    }
    u64* o = out + (size_t)blockIdx.x * 3 * P + (size_t)limb * N + x;
    if (SPLIT) {
        o[0] = acc3_reduce(t00, 20, m);
        o[P] = acc3_reduce(t01, 20, m);
        o[2 * P] = acc3_reduce(t11, 20, m);
    } else {
        o[0] = reduce128(s00, m);
        o[P] = reduce128(s01, m);
        o[2 * P] = reduce128(s11, m);
    }
}

// ---------------------------------------------------------------------------- device randomness
// Philox4x64-10 (Salmon et al., SC 2011) from its definition; sampling rules: key = (seed, 0),
// counter = (coefficient, ciphertext index, purpose, 0); ternary r from the top 32 bits of word 0
// by multiply-shift; errors centred binomial with eta = 21 from words 0 and 1.
__device__ __forceinline__ void philox4x64_10(u64& x0, u64& x1, u64& x2, u64& x3, u64 k0, u64 k1) {
    const u64 M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const u64 W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; r++) {
        if (r) {
            k0 += W0;
            k1 += W1;
        }
        const u64 hi0 = __umul64hi(M0, x0), lo0 = M0 * x0;
        const u64 hi1 = __umul64hi(M1, x2), lo1 = M1 * x2;
        const u64 y0 = hi1 ^ x1 ^ k0, y2 = hi0 ^ x3 ^ k1;
        x0 = y0;
        x1 = lo1;
        x2 = y2;
        x3 = lo0;
    }
}

__global__ void k_sample_enc(u64 seed, u64 first, int count, int log_n, int8_t* __restrict__ r,
                             int32_t* __restrict__ e0, int32_t* __restrict__ e1) {
    const size_t N = (size_t)1 << log_n;
    const size_t total = (size_t)count * N;
    const u64 m21 = (1ull << 21) - 1;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const u64 k = i & (N - 1), c = first + (i >> log_n);
        u64 a = k, b = c, d = 0, e = 0;
        philox4x64_10(a, b, d, e, seed, 0);
        r[i] = (int8_t)((int)(((a >> 32) * 3) >> 32) - 1);
        a = k, b = c, d = 1, e = 0;
        philox4x64_10(a, b, d, e, seed, 0);
        e0[i] = __popcll(a & m21) - __popcll(b & m21);
        a = k, b = c, d = 2, e = 0;
        philox4x64_10(a, b, d, e, seed, 0);
        e1[i] = __popcll(a & m21) - __popcll(b & m21);
    }
}

// constant-slot plaintexts: m[b] = (round(w[b] * scale), 0, ..., 0)
__global__ void k_const_plain(const double* __restrict__ w, int count, int log_n, double scale,
                              int64_t* __restrict__ m) {
    const size_t N = (size_t)1 << log_n;
    const size_t total = (size_t)count * N;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x)
        m[i] = (i & (N - 1)) ? 0 : __double2ll_rn(w[i >> log_n] * scale);
}

// ---------------------------------------------------------------------------- KGC step on the device
// read-out values: centred residue mod q0 divided by the scale
__global__ void k_readout_finish(const u64* __restrict__ res, int count, const ModConst* __restrict__ mc,
                                 double scale, double* __restrict__ out) {
    const u64 q0 = mc[0].q;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < count; b += gridDim.x * blockDim.x) {
        const u64 v = res[b];
        out[b] = (v > q0 / 2 ? -(double)(q0 - v) : (double)v) / scale;
    }
}

// Krum / Multi-Krum (Algorithm 2) on n <= 256 clients from the pair distances d (i < j,
// lexicographic): score_i = sum of the n - f - 2 smallest d(i, j), j != i; the l lowest scores are
// kept (stable: ties go to the lower index); w_i = 1 / l (average) or 1 for kept clients, else 0.
// One block of at least n threads.
__global__ void k_krum(const double* __restrict__ d, int n, int f, int l, int average, double* __restrict__ w,
                       int* __restrict__ sel) {
    __shared__ double score[256];
    const int i = threadIdx.x;
    const int k = max(0, n - f - 2);
    if (i < n) {
        // the k smallest of row i by repeated minimum (n <= 256, k < n): ascending order, summed
        // in that order
        double last = -1.0;
        int last_j = -1;
        double sum = 0.0;
        for (int t = 0; t < k; t++) {
            double best = 0.0;
            int bj = -1;
            for (int j = 0; j < n; j++) {
                if (j == i) continue;
                const int a = min(i, j), b = max(i, j);
                const double v = d[a * n - a * (a + 1) / 2 + (b - a - 1)];
                // strictly after (last, last_j) in (value, index) order
                const bool after = v > last || (v == last && j > last_j);
                if (after && (bj < 0 || v < best || (v == best && j < bj))) {
                    best = v;
                    bj = j;
                }
            }
            sum += best;
            last = best;
            last_j = bj;
        }
        score[i] = sum;
        w[i] = 0.0;
    }
    __syncthreads();
    if (i == 0) {
        int lastc = -1;
        double lasts = 0.0;
        for (int t = 0; t < l; t++) {
            int bc = -1;
            double bs = 0.0;
            for (int c2 = 0; c2 < n; c2++) {
                const double v = score[c2];
                const bool after = lastc < 0 || v > lasts || (v == lasts && c2 > lastc);
                if (after && (bc < 0 || v < bs)) {
                    bs = v;
                    bc = c2;
                }
            }
            sel[t] = bc;
            w[bc] = average ? 1.0 / l : 1.0;
            lastc = bc;
            lasts = bs;
        }
    }
}

// ---------------------------------------------------------------------------- encoding (FP64)
// Canonical-embedding encode of real slot vectors (Section "CKKS Scheme Description"):
//   A[5^j mod 2N] = scale z_j (j < N/2, other entries 0), X = FFT_2N(A) with e^{-2 pi i/2N},
//   m_k = round(2/N Re X_k) for k < N  (ties to even).
// The 2N-point FFT is done as 256 x (2N/256) four-step: column FFTs of length 256 over the high
// index bits with the twist e^{-2 pi i t2 k1 / 2N}, then row FFTs over the low bits.
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ unsigned brev8(unsigned v) { return __brev(v) >> 24; }

// in-place radix-2 FFT of NF interleaved 256-point sequences s[f][256] (bit-reversed input,
// natural output), 128 threads
template <int NF>
__device__ __forceinline__ void fft256_block(double2 (*s)[256], const double2* __restrict__ w256) {
    for (int len = 2; len <= 256; len <<= 1) {
        const int half = len >> 1, step = 256 / len;
        for (int b = threadIdx.x; b < 128 * NF; b += 128) {
            const int f = b >> 7, bb = b & 127;
            const int grp = bb / half, pos = bb - grp * half;
            const int i = grp * len + pos, j = i + half;
            const double2 u = s[f][i], v = cmul(s[f][j], __ldg(w256 + pos * step));
            s[f][i] = make_double2(u.x + v.x, u.y + v.y);
            s[f][j] = make_double2(u.x - v.x, u.y - v.y);
        }
        __syncthreads();
    }
}

// A[b][2N] <- 0, then A[b][pos[j]] = (scale z[b][j], 0)
__global__ void k_enc_scatter(const double* __restrict__ z, int count, int log_n, const unsigned* __restrict__ pos,
                              double scale, double2* __restrict__ A) {
    const size_t N = (size_t)1 << log_n, half = N / 2;
    const size_t total = (size_t)count * half;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t b = i / half, j = i - b * half;
        A[b * 2 * N + pos[j]] = make_double2(scale * z[i], 0.0);
    }
}

// column pass: 8 columns t2 per block; x[t1][t2] with t1 < 256 -> Y[k1][t2] = FFT_t1 * w^{t2 k1}
__global__ void __launch_bounds__(128) k_fft_cols(double2* __restrict__ A, int log_2n, const double2* __restrict__ w256,
                                                  const double2* __restrict__ wbig) {
    __shared__ double2 s[8][256];
    const size_t M = (size_t)1 << log_2n, cols = M >> 8;
    double2* a = A + (size_t)blockIdx.y * M;
    const int c0 = blockIdx.x * 8;
    for (int e = threadIdx.x; e < 2048; e += 128) {
        const int t1 = e >> 3, c = e & 7;
        s[c][brev8(t1)] = a[(size_t)t1 * cols + c0 + c];
    }
    __syncthreads();
    fft256_block<8>(s, w256);
    for (int e = threadIdx.x; e < 2048; e += 128) {
        const int k1 = e >> 3, c = e & 7;
        a[(size_t)k1 * cols + c0 + c] = cmul(s[c][k1], __ldg(wbig + (size_t)(c0 + c) * k1));
    }
}

// row pass for 2N = 256 * 256 (log_n = 15): 8 rows k1 per block, FFT over t2, output
// m[k1 + 256 k2] = round(2/N Re X) for k2 < N / 256
__global__ void __launch_bounds__(128) k_fft_rows_out(const double2* __restrict__ A, int log_n,
                                                      const double2* __restrict__ w256, int64_t* __restrict__ m) {
    __shared__ double2 s[8][256];
    const size_t N = (size_t)1 << log_n, M = 2 * N, cols = M >> 8;  // cols = 256 here
    const double2* a = A + (size_t)blockIdx.y * M;
    int64_t* mb = m + (size_t)blockIdx.y * N;
    const int r0 = blockIdx.x * 8;
    for (int e = threadIdx.x; e < 2048; e += 128) {
        const int r = e >> 8, t2 = e & 255;
        s[r][brev8(t2)] = a[(size_t)(r0 + r) * cols + t2];
    }
    __syncthreads();
    fft256_block<8>(s, w256);
    const double f = 2.0 / (double)N;
    const int k2max = (int)(N >> 8);
    for (int e = threadIdx.x; e < 8 * k2max; e += 128) {
        const int k2 = e >> 3, r = e & 7;
        mb[(size_t)(r0 + r) + 256 * (size_t)k2] = __double2ll_rn(f * s[r][k2].x);
    }
}

// group-kernel key layout: rows (of all n_q + n_p) with primes below 2^40 as packed halves
__global__ void k_pack_key(const u64* __restrict__ in, u64* __restrict__ out, int rows, int log_n,
                           const ModConst* __restrict__ mc, size_t total) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int m = (int)((i >> log_n) % rows);
        const u64 v = in[i];
        out[i] = mc[m].q < (1ull << 40) ? (((v >> 20) << 32) | (v & 0xFFFFFu)) : v;
    }
}

// ---------------------------------------------------------------------------- multi-job items
// masked accumulate of one chunk of one job per item.  grid: x = item, y = tile, z = limb
template <bool SPLIT>
__global__ void __launch_bounds__(kT) k_mask_acc_items(const AggItem* __restrict__ items, int nl, int limb0,
                                                       int log_n, const ModConst* __restrict__ mc,
                                                       u64* __restrict__ out) {
    const AggItem it = items[blockIdx.x];
    const int limb = limb0 + blockIdx.z;
    const size_t N = (size_t)1 << log_n;
    const size_t x = (size_t)blockIdx.y * kT + threadIdx.x;
    const ModConst m = mc[limb];
    const size_t P = (size_t)nl * N;
    u128v s00{0, 0}, s01{0, 0}, s11{0, 0};
    Acc3 t00{0, 0, 0}, t01{0, 0, 0}, t11{0, 0, 0};
    for (int i = 0; i < it.n; i++) {
        const u64* a = it.cts + ((size_t)i * it.chunks + it.k) * 2 * P + (size_t)limb * N + x;
        const u64* w = it.masks + (size_t)i * 2 * P + (size_t)limb * N + x;
        const u64 a0 = __ldg(a), a1 = __ldg(a + P), m0 = __ldg(w), m1 = __ldg(w + P);
        if (SPLIT) {
            const unsigned ah0 = (unsigned)(a0 >> 20), al0 = (unsigned)a0 & 0xFFFFFu;
            const unsigned ah1 = (unsigned)(a1 >> 20), al1 = (unsigned)a1 & 0xFFFFFu;
            const unsigned mh0 = (unsigned)(m0 >> 20), ml0 = (unsigned)m0 & 0xFFFFFu;
            const unsigned mh1 = (unsigned)(m1 >> 20), ml1 = (unsigned)m1 & 0xFFFFFu;
            mac_split(t00, ah0, al0, mh0, ml0);
            mac_split(t01, ah0, al0, mh1, ml1);
            mac_split(t01, ah1, al1, mh0, ml0);
            mac_split(t11, ah1, al1, mh1, ml1);
        } else {
            mac128(s00, a0, m0);
            mac128(s01, a0, m1);
            mac128(s01, a1, m0);
            mac128(s11, a1, m1);
            if ((i & 3) == 3) {
                fold(s00, m);
                fold(s01, m);
                fold(s11, m);
            }
        }
    }
    u64* o = out + (size_t)it.slot * 3 * P + (size_t)limb * N + x;
    o[0] = SPLIT ? acc3_reduce(t00, 20, m) : reduce128(s00, m);
    o[P] = SPLIT ? acc3_reduce(t01, 20, m) : reduce128(s01, m);
    o[2 * P] = SPLIT ? acc3_reduce(t11, 20, m) : reduce128(s11, m);
}

// words-per-item copy to per-item destinations.  grid: x = chunk of 2*kT words, y = item
__global__ void k_copy_items(const u64* __restrict__ src, size_t words, u64* const* __restrict__ dst) {
    const int b = blockIdx.y;
    u64* d = dst[b];
    const u64* s = src + (size_t)b * words;
    for (size_t i = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) * 2; i < words; i += (size_t)gridDim.x * blockDim.x * 2) {
        const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(s + i);
        *reinterpret_cast<ulonglong2*>(d + i) = v;
    }
}

// KGC read-out of ciphertexts that hold one value in every slot: coefficient 0 of c0 + c1 s
// mod q0, i.e. N^-1 * sum_idx (c0 + c1 s)[idx] over the evaluation-domain limb 0.
// grid: x = ciphertext; block reduction of 128-bit partial sums.
__global__ void __launch_bounds__(kT) k_const_coef0(const u64* __restrict__ cts, size_t ct_stride,
                                                   const u64* __restrict__ s0, int log_n,
                                                   const ModConst* __restrict__ mc, u64* __restrict__ out) {
    __shared__ u64 red[kT];
    const ModConst m = mc[0];
    const size_t N = (size_t)1 << log_n;
    const size_t P = ct_stride / 2;  // words per polynomial
    const u64* c0 = cts + (size_t)blockIdx.x * ct_stride;
    const u64* c1 = c0 + P;
    u128v acc{0, 0};
    for (size_t i = threadIdx.x; i < N; i += kT) {
        const u64 v = add_mod(c0[i], mul_mod(c1[i], s0[i], m), m.q);
        add128(acc, v);
    }
    red[threadIdx.x] = reduce128(acc, m);
    __syncthreads();
    for (int w = kT / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] = add_mod(red[threadIdx.x], red[threadIdx.x + w], m.q);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = mul_shoup(red[0], m.n_inv, m.n_inv_sh, m.q);
}

// ---------------------------------------------------------------------------- base conversion
// All four kernels handle VEC consecutive coefficients per thread with 16-byte accesses; the
// per-destination reduction constants come from the shared-memory copy of the table.

template <typename Tab>
__device__ __forceinline__ void load_tab(Tab& dst, const Tab* src) {
    const int words = sizeof(Tab) / 8;
    const u64* s = reinterpret_cast<const u64*>(src);
    u64* d = reinterpret_cast<u64*>(&dst);
    for (int w = threadIdx.x; w < words; w += blockDim.x) d[w] = s[w];
    __syncthreads();
}

__device__ __forceinline__ ulonglong2 ld2(const u64* p) { return __ldg(reinterpret_cast<const ulonglong2*>(p)); }
__device__ __forceinline__ void st2(u64* p, u64 a, u64 b) { *reinterpret_cast<ulonglong2*>(p) = make_ulonglong2(a, b); }

// ModUp of NS-prime digits j0 .. j0+nj-1.  grid: x = tile of 2*kT coefficients, y = b * nj + (j - j0)
template <int NS>
__global__ void __launch_bounds__(kT) k_modup(const u64* __restrict__ coef, size_t coef_stride, int beta, int j0,
                                              int nj, int rows, int log_n, const ModUpTab* __restrict__ tabs,
                                              u64* __restrict__ ext) {
    __shared__ ModUpTab tab;
    const int b = blockIdx.y / nj, j = j0 + (blockIdx.y - (blockIdx.y / nj) * nj);
    load_tab(tab, tabs + j);
    const size_t N = (size_t)1 << log_n;
    const size_t x = ((size_t)blockIdx.x * kT + threadIdx.x) * 2;
    const u64* cb = coef + (size_t)b * coef_stride + x;
    u64 y0[NS], y1[NS];
    unsigned negm = 0;
#pragma unroll
    for (int i = 0; i < NS; i++) {
        const u64 q = tab.src_q[i];
        const ulonglong2 v = ld2(cb + ((size_t)tab.src_row[i] << log_n));
        y0[i] = csub(mul_shoup_lazy(v.x, tab.hinv[i], tab.hinv_sh[i], q), q);
        y1[i] = csub(mul_shoup_lazy(v.y, tab.hinv[i], tab.hinv_sh[i], q), q);
        negm |= (y0[i] > (q >> 1) ? 1u : 0u) << (2 * i);
        negm |= (y1[i] > (q >> 1) ? 2u : 0u) << (2 * i);
    }
    u64* eb = ext + ((size_t)b * beta + j) * rows * N + x;
    const int nd = tab.n_dst;
#pragma unroll 2
    for (int t = 0; t < nd; t++) {
        u128v a0{0, 0}, a1{0, 0};
#pragma unroll
        for (int i = 0; i < NS; i++) {
            const u64 h = tab.hat[i][t], cr = tab.corr[i][t];
            mac128(a0, y0[i], h);
            mac128(a1, y1[i], h);
            if (negm >> (2 * i) & 1) add128(a0, cr);
            if (negm >> (2 * i) & 2) add128(a1, cr);
        }
        const u64 q = tab.dq[t], r64 = tab.dr64[t], r64sh = tab.dr64sh[t], osh = tab.donesh[t];
        st2(eb + ((size_t)tab.dst_row[t] << log_n), reduce128c(a0, q, r64, r64sh, osh),
            reduce128c(a1, q, r64, r64sh, osh));
    }
}

// key inner product.  grid: x = batch item (fastest: one key tile serves every item through L2),
// y = tile of 4*kT coefficients, z = row t of Q_l U P
__global__ void __launch_bounds__(kT) k_inner(const u64* __restrict__ ext, const u64* __restrict__ d, size_t d_stride,
                                              int beta, int nl, int rows, int alpha, int nq, int nqp, int log_n,
                                              const u64* __restrict__ key, const ModConst* __restrict__ mc,
                                              u64* __restrict__ v) {
    const int b = blockIdx.x, t = blockIdx.z;
    const size_t N = (size_t)1 << log_n;
    const size_t x = ((size_t)blockIdx.y * kT + threadIdx.x) * 4;
    const int kt = t < nl ? t : nq + (t - nl);
    const ModConst& mcr = mc[kt];
    const u64 q = __ldg(&mcr.q), r64 = __ldg(&mcr.r64), r64sh = __ldg(&mcr.r64_sh), osh = __ldg(&mcr.one_sh);
    u128v a[4], c[4];
#pragma unroll
    for (int k = 0; k < 4; k++) a[k] = c[k] = u128v{0, 0};
    for (int j = 0; j < beta; j++) {
        const u64* src = (t < nl && t / alpha == j) ? d + (size_t)b * d_stride + ((size_t)t << log_n)
                                                     : ext + (((size_t)b * beta + j) * rows + t) * N;
        const u64* kb = key + (((size_t)j * 2 + 0) * nqp + kt) * N + x;
        const u64* ka = key + (((size_t)j * 2 + 1) * nqp + kt) * N + x;
        const ulonglong2 e01 = ld2(src + x), e23 = ld2(src + x + 2);
        const ulonglong2 b01 = ld2(kb), b23 = ld2(kb + 2), a01 = ld2(ka), a23 = ld2(ka + 2);
        mac128(a[0], e01.x, b01.x);
        mac128(a[1], e01.y, b01.y);
        mac128(a[2], e23.x, b23.x);
        mac128(a[3], e23.y, b23.y);
        mac128(c[0], e01.x, a01.x);
        mac128(c[1], e01.y, a01.y);
        mac128(c[2], e23.x, a23.x);
        mac128(c[3], e23.y, a23.y);
    }
    u64* vb = v + (size_t)b * 2 * rows * N + (size_t)t * N + x;
    st2(vb, reduce128c(a[0], q, r64, r64sh, osh), reduce128c(a[1], q, r64, r64sh, osh));
    st2(vb + 2, reduce128c(a[2], q, r64, r64sh, osh), reduce128c(a[3], q, r64, r64sh, osh));
    u64* vc = vb + (size_t)rows * N;
    st2(vc, reduce128c(c[0], q, r64, r64sh, osh), reduce128c(c[1], q, r64, r64sh, osh));
    st2(vc + 2, reduce128c(c[2], q, r64, r64sh, osh), reduce128c(c[3], q, r64, r64sh, osh));
}

// key inner product for T keys of one hoisted group, reading the extended digits once:
// v_t = sum_j E_j * key_t,j for t < T.  keys: device array of T key pointers.
// grid: x = batch item, y = tile of 2*kT coefficients, z = row t of Q_l U P
template <int T>
__global__ void __launch_bounds__(kT) k_inner_multi(const u64* __restrict__ ext, const u64* __restrict__ d,
                                                    size_t d_stride, int beta, int nl, int rows, int alpha, int nq,
                                                    int nqp, int log_n, KeyPtrs keys, const ModConst* __restrict__ mc,
                                                    u64* __restrict__ v, size_t v_key_stride) {
    const int b = blockIdx.x, t = blockIdx.z;
    const size_t N = (size_t)1 << log_n;
    const size_t x = ((size_t)blockIdx.y * kT + threadIdx.x) * 2;
    const int kt = t < nl ? t : nq + (t - nl);
    const ModConst& mcr = mc[kt];
    const u64 q = __ldg(&mcr.q), r64 = __ldg(&mcr.r64), r64sh = __ldg(&mcr.r64_sh), osh = __ldg(&mcr.one_sh);
    u128v a[T][2], c[T][2];
#pragma unroll
    for (int k = 0; k < T; k++) a[k][0] = a[k][1] = c[k][0] = c[k][1] = u128v{0, 0};
    for (int j = 0; j < beta; j++) {
        const u64* src = (t < nl && t / alpha == j) ? d + (size_t)b * d_stride + ((size_t)t << log_n)
                                                     : ext + (((size_t)b * beta + j) * rows + t) * N;
        const ulonglong2 e = ld2(src + x);
        const size_t ko = (((size_t)j * 2 + 0) * nqp + kt) * N + x;
        const size_t ka = (size_t)nqp * N;
#pragma unroll
        for (int k = 0; k < T; k++) {
            const ulonglong2 kb2 = ld2(keys.p[k] + ko), ka2 = ld2(keys.p[k] + ko + ka);
            mac128(a[k][0], e.x, kb2.x);
            mac128(a[k][1], e.y, kb2.y);
            mac128(c[k][0], e.x, ka2.x);
            mac128(c[k][1], e.y, ka2.y);
        }
    }
#pragma unroll
    for (int k = 0; k < T; k++) {
        u64* vb = v + k * v_key_stride + (size_t)b * 2 * rows * N + (size_t)t * N + x;
        st2(vb, reduce128c(a[k][0], q, r64, r64sh, osh), reduce128c(a[k][1], q, r64, r64sh, osh));
        st2(vb + (size_t)rows * N, reduce128c(c[k][0], q, r64, r64sh, osh), reduce128c(c[k][1], q, r64, r64sh, osh));
    }
}

// same as k_inner_multi with per-item keys: keys[b * T + t]
template <int T>
__global__ void __launch_bounds__(kT) k_inner_items(const u64* __restrict__ ext, const u64* __restrict__ d,
                                                    size_t d_stride, int beta, int nl, int rows, int alpha, int nq,
                                                    int nqp, int log_n, const u64* const* __restrict__ keys,
                                                    const ModConst* __restrict__ mc, u64* __restrict__ v,
                                                    size_t v_key_stride) {
    const int b = blockIdx.x, t = blockIdx.z;
    const size_t N = (size_t)1 << log_n;
    const size_t x = ((size_t)blockIdx.y * kT + threadIdx.x) * 2;
    const int kt = t < nl ? t : nq + (t - nl);
    const ModConst& mcr = mc[kt];
    const u64 q = __ldg(&mcr.q), r64 = __ldg(&mcr.r64), r64sh = __ldg(&mcr.r64_sh), osh = __ldg(&mcr.one_sh);
    const u64* kp[T];
#pragma unroll
    for (int k = 0; k < T; k++) kp[k] = keys[(size_t)b * T + k];
    u128v a[T][2], c[T][2];
#pragma unroll
    for (int k = 0; k < T; k++) a[k][0] = a[k][1] = c[k][0] = c[k][1] = u128v{0, 0};
    for (int j = 0; j < beta; j++) {
        const u64* src = (t < nl && t / alpha == j) ? d + (size_t)b * d_stride + ((size_t)t << log_n)
                                                     : ext + (((size_t)b * beta + j) * rows + t) * N;
        const ulonglong2 e = ld2(src + x);
        const size_t ko = (((size_t)j * 2 + 0) * nqp + kt) * N + x;
        const size_t ka = (size_t)nqp * N;
#pragma unroll
        for (int k = 0; k < T; k++) {
            const ulonglong2 kb2 = ld2(kp[k] + ko), ka2 = ld2(kp[k] + ko + ka);
            mac128(a[k][0], e.x, kb2.x);
            mac128(a[k][1], e.y, kb2.y);
            mac128(c[k][0], e.x, ka2.x);
            mac128(c[k][1], e.y, ka2.y);
        }
    }
#pragma unroll
    for (int k = 0; k < T; k++) {
        u64* vb = v + k * v_key_stride + (size_t)b * 2 * rows * N + (size_t)t * N + x;
        st2(vb, reduce128c(a[k][0], q, r64, r64sh, osh), reduce128c(a[k][1], q, r64, r64sh, osh));
        st2(vb + (size_t)rows * N, reduce128c(c[k][0], q, r64, r64sh, osh), reduce128c(c[k][1], q, r64, r64sh, osh));
    }
}

// usum[p][r][idx] = sum_t src_t[p][r][perm_{g_t}(idx)] over polys of `rows` rows (Q_l U P)
template <int T>
__global__ void k_gather_sum(const u64* __restrict__ src, size_t src_stride, u64* __restrict__ usum, int n_polys,
                             int rows, int nlq, int nq, int log_n, Galois gs, const ModConst* __restrict__ mc) {
    const size_t N = (size_t)1 << log_n;
    const size_t total = (size_t)n_polys * rows * N;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
        const unsigned x = (unsigned)(idx & (N - 1));
        const size_t row = idx >> log_n;
        const int r = (int)(row % rows);
        const u64 q = mc[r < nlq ? r : nq + (r - nlq)].q;
        u64 acc = 0;
#pragma unroll
        for (int k = 0; k < T; k++) acc = add_mod(acc, src[k * src_stride + (row << log_n) + auto_src(x, gs.g[k], log_n)], q);
        usum[idx] = acc;
    }
}

// One hoisted group with a single ModDown, fused: for the T rotations g_t of the group,
//   usum[b][p][r][x]  = sum_t sum_j E_j[b][r][s_t] * k'_t[j][p][r][s_t],   s_t = perm_{g_t}(x)
//   c0acc[b][r][x]    = y0[b][r][x] + sum_t y0[b][r][s_t]                    (rows r < nl)
// i.e. sum_t phi_{g_t}(<E, k'_t>) with k'_t the keys pre-permuted by phi_{g_t}^-1, without
// writing the per-rotation products.  k'_t[s_t(x)] is the un-permuted key at x, so the keys are
// read in their group-kernel layout (SwKey::qp: un-permuted, 40-bit rows as packed halves).  E_j is the j-th extended digit (own rows from d).  All
// products of one output sum in 128 bits (T * beta < 64 terms below q^2 < 2^120) and reduce
// once, so the result equals the per-rotation reduction exactly.
// perm_g maps the aligned pair {2m, 2m+1} onto an aligned pair {s, s^1} (the pair bit is the top
// bit of the bit-reversed index, and X -> X^g adds an odd multiple of 2^(log_n-1) to it), so a
// thread owns two coefficients and every gather is one 16-byte load plus a conditional swap.
// grid: x = group of kBT items (fastest, so that consecutive blocks share the key tile in L2),
// y = tile of 2 kTG coefficients, z = row r of Q_l U P.
constexpr int kTG = 128;
__device__ __forceinline__ ulonglong2 ld2_swap(const u64* p, unsigned s0, bool sw) {
    const ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2*>(p + s0));
    return sw ? make_ulonglong2(v.y, v.x) : v;
}
// the rows (of Q_l U P) one launch covers: [a0, a0 + na) then [b0, ...), in blockIdx.z order
struct RowSel {
    int a0, na, b0;
};
// SPLIT: every selected row's prime is below 2^40, so digits and keys split into 20-bit halves
// (four 32x32 -> 64-bit products per 128-bit product, three 64-bit partial sums).
// KARA (with SPLIT): three products instead of four -- h h', l l' and (h + l)(h' + l'), whose
// sum minus the other two is the middle term h l' + l h' (Karatsuba); every term is a
// non-negative integer, (h + l)(h' + l') < 2^42 and at most 60 of them are summed, so the
// partial sums stay below 2^48 and the result is the same integer.
// Register caps with one item per thread: 4 resident blocks for the split rows (128 registers;
// 5 blocks: 96 registers and 1.5 % slower, 3 blocks: 6 % slower), 3 for the 128-bit ones (164-168
// registers instead of 208, no spills: 4 % faster than uncapped).
template <int T, bool ITEMS, bool SPLIT, int kBT, bool KARA = false>
__global__ void __launch_bounds__(kTG, kBT == 1 ? (SPLIT ? 4 : 3) : 1) k_inner_gather(const u64* __restrict__ ext, const u64* __restrict__ d,
                                                     size_t d_stride, const u64* __restrict__ y0, size_t y0_stride,
                                                     int B, int beta, int nl, int rows, int alpha, int nq, int nqp,
                                                     int log_n, KeyPtrs keys, const u64* const* __restrict__ keys_dev,
                                                     Galois gs, RowSel sel, const ModConst* __restrict__ mc,
                                                     u64* __restrict__ usum, u64* __restrict__ c0acc) {
    const size_t N = (size_t)1 << log_n;
    const unsigned x = (blockIdx.y * kTG + threadIdx.x) * 2;
    const int z = blockIdx.z;
    const int r = z < sel.na ? sel.a0 + z : sel.b0 + (z - sel.na);
    const int b0 = blockIdx.x * kBT;
    const int nb = min(kBT, B - b0);
    const int kt = r < nl ? r : nq + (r - nl);
    const ModConst& mcr = mc[kt];
    const u64 q = __ldg(&mcr.q), r64 = __ldg(&mcr.r64), r64sh = __ldg(&mcr.r64_sh), osh = __ldg(&mcr.one_sh);
    unsigned s0[T];
    bool sw[T];
#pragma unroll
    for (int t = 0; t < T; t++) {
        const unsigned sv = auto_src(x, gs.g[t], log_n);
        s0[t] = sv & ~1u;
        sw[t] = sv & 1u;
    }
    // items past the end of the batch repeat the last one; their results are not stored
    int bi[kBT];
#pragma unroll
    for (int i = 0; i < kBT; i++) bi[i] = b0 + min(i, nb - 1);
    u128v a[SPLIT ? 1 : kBT][2][2];
    Acc3 h[SPLIT ? kBT : 1][2][2];
#pragma unroll
    for (int i = 0; i < kBT; i++) {
        if (SPLIT)
            h[i][0][0] = h[i][0][1] = h[i][1][0] = h[i][1][1] = Acc3{0, 0, 0};
        else
            a[i][0][0] = a[i][0][1] = a[i][1][0] = a[i][1][1] = u128v{0, 0};
    }
    const size_t ka = (size_t)nqp * N;
    for (int j = 0; j < beta; j++) {
        const bool own = r < nl && r / alpha == j;
        const size_t ko = ((size_t)j * 2 * nqp + kt) * N;
#pragma unroll
        for (int t = 0; t < T; t++) {
            // keys in the group-kernel layout: read at x (no permutation), 40-bit rows packed
            ulonglong2 k0, k1;
            if (!ITEMS) {
                k0 = ld2(keys.p[t] + ko + x);
                k1 = ld2(keys.p[t] + ko + ka + x);
            }
#pragma unroll
            for (int i = 0; i < kBT; i++) {
                const int b = bi[i];
                if (ITEMS) {
                    const u64* kp = keys_dev[(size_t)b * T + t];
                    k0 = ld2(kp + ko + x);
                    k1 = ld2(kp + ko + ka + x);
                }
                const u64* e = own ? d + (size_t)b * d_stride + ((size_t)r << log_n)
                                   : ext + (((size_t)b * beta + j) * rows + r) * N;
                const ulonglong2 ev = ld2_swap(e, s0[t], sw[t]);
                if (SPLIT && KARA) {
                    const unsigned exh = (unsigned)(ev.x >> 20), exl = (unsigned)ev.x & 0xFFFFFu;
                    const unsigned eyh = (unsigned)(ev.y >> 20), eyl = (unsigned)ev.y & 0xFFFFFu;
                    mac_kara(h[i][0][0], exh, exl, exh + exl, (unsigned)(k0.x >> 32), (unsigned)k0.x);
                    mac_kara(h[i][0][1], eyh, eyl, eyh + eyl, (unsigned)(k0.y >> 32), (unsigned)k0.y);
                    mac_kara(h[i][1][0], exh, exl, exh + exl, (unsigned)(k1.x >> 32), (unsigned)k1.x);
                    mac_kara(h[i][1][1], eyh, eyl, eyh + eyl, (unsigned)(k1.y >> 32), (unsigned)k1.y);
                } else if (SPLIT) {
                    const unsigned exh = (unsigned)(ev.x >> 20), exl = (unsigned)ev.x & 0xFFFFFu;
                    const unsigned eyh = (unsigned)(ev.y >> 20), eyl = (unsigned)ev.y & 0xFFFFFu;
                    mac_split(h[i][0][0], exh, exl, (unsigned)(k0.x >> 32), (unsigned)k0.x);
                    mac_split(h[i][0][1], eyh, eyl, (unsigned)(k0.y >> 32), (unsigned)k0.y);
                    mac_split(h[i][1][0], exh, exl, (unsigned)(k1.x >> 32), (unsigned)k1.x);
                    mac_split(h[i][1][1], eyh, eyl, (unsigned)(k1.y >> 32), (unsigned)k1.y);
                } else {
                    mac128(a[i][0][0], ev.x, k0.x);
                    mac128(a[i][0][1], ev.y, k0.y);
                    mac128(a[i][1][0], ev.x, k1.x);
                    mac128(a[i][1][1], ev.y, k1.y);
                }
            }
        }
    }
#pragma unroll
    for (int i = 0; i < kBT; i++) {
        if (i < nb) {
            const int b = b0 + i;
            u64* ub = usum + ((size_t)b * 2 * rows + r) * N + x;
            if (SPLIT) {
                if (KARA) {  // middle terms: sum (h + l)(h' + l') - sum h h' - sum l l'
#pragma unroll
                    for (int p2 = 0; p2 < 2; p2++)
#pragma unroll
                        for (int c2 = 0; c2 < 2; c2++) h[i][p2][c2].b -= h[i][p2][c2].a + h[i][p2][c2].c;
                }
                st2(ub, acc3_reduce(h[i][0][0], 20, mcr), acc3_reduce(h[i][0][1], 20, mcr));
                st2(ub + (size_t)rows * N, acc3_reduce(h[i][1][0], 20, mcr), acc3_reduce(h[i][1][1], 20, mcr));
            } else {
                st2(ub, reduce128c(a[i][0][0], q, r64, r64sh, osh), reduce128c(a[i][0][1], q, r64, r64sh, osh));
                st2(ub + (size_t)rows * N, reduce128c(a[i][1][0], q, r64, r64sh, osh),
                    reduce128c(a[i][1][1], q, r64, r64sh, osh));
            }
            if (r < nl) {
                const u64* yb = y0 + (size_t)b * y0_stride + ((size_t)r << log_n);
                const ulonglong2 self = ld2(yb + x);
                u64 c0 = self.x, c1 = self.y;  // T + 1 < 16 terms below q < 2^60
#pragma unroll
                for (int t = 0; t < T; t++) {
                    const ulonglong2 v = ld2_swap(yb, s0[t], sw[t]);
                    c0 += v.x;
                    c1 += v.y;
                }
                st2(c0acc + ((size_t)b * nl + r) * N + x, reduce64(c0, mcr), reduce64(c1, mcr));
            }
        }
    }
}

// ModDown conversion of the K special-prime rows.  grid: x = tile of 2*kT coefficients, y = b*2 + k
template <int K>
__global__ void __launch_bounds__(kT) k_moddown_bconv(const u64* __restrict__ v, int nl, int rows, int log_n,
                                                      const ModDownTab* __restrict__ tabp, u64* __restrict__ conv) {
    __shared__ ModDownTab tab;
    load_tab(tab, tabp);
    const size_t N = (size_t)1 << log_n;
    const size_t x = ((size_t)blockIdx.x * kT + threadIdx.x) * 2;
    const int bk = blockIdx.y;
    const u64* vb = v + (size_t)bk * rows * N + x;
    u64 y0[K], y1[K];
    unsigned negm = 0;
#pragma unroll
    for (int k = 0; k < K; k++) {
        const u64 p = tab.p[k];
        const ulonglong2 val = ld2(vb + ((size_t)(nl + k) << log_n));
        y0[k] = csub(mul_shoup_lazy(val.x, tab.phinv[k], tab.phinv_sh[k], p), p);
        y1[k] = csub(mul_shoup_lazy(val.y, tab.phinv[k], tab.phinv_sh[k], p), p);
        negm |= (y0[k] > (p >> 1) ? 1u : 0u) << (2 * k);
        negm |= (y1[k] > (p >> 1) ? 2u : 0u) << (2 * k);
    }
    u64* cb = conv + (size_t)bk * nl * N + x;
#pragma unroll 2
    for (int i = 0; i < nl; i++) {
        u128v a0{0, 0}, a1{0, 0};
#pragma unroll
        for (int k = 0; k < K; k++) {
            const u64 h = tab.phat[k][i], cr = tab.corr[k][i];
            mac128(a0, y0[k], h);
            mac128(a1, y1[k], h);
            if (negm >> (2 * k) & 1) add128(a0, cr);
            if (negm >> (2 * k) & 2) add128(a1, cr);
        }
        const u64 q = tab.qq[i], r64 = tab.qr64[i], r64sh = tab.qr64sh[i], osh = tab.qonesh[i];
        st2(cb + ((size_t)i << log_n), reduce128c(a0, q, r64, r64sh, osh), reduce128c(a1, q, r64, r64sh, osh));
    }
}

// W[b][k] = (v_k - conv_k) P^-1 + add_k over 2 coefficients per thread; grid-stride over B*2*nl*N/2
__global__ void k_moddown_combine(const u64* __restrict__ v, const u64* __restrict__ conv, int B, int nl, int rows,
                                  int log_n, const ModDownTab* __restrict__ tab, const ModConst* __restrict__ mc,
                                  const u64* add0, size_t add0_stride, const u64* add1, size_t add1_stride,
                                  u64* w, size_t w_stride) {
    const size_t N = (size_t)1 << log_n;
    const size_t total = (size_t)B * 2 * nl * N / 2;
    for (size_t h = (size_t)blockIdx.x * blockDim.x + threadIdx.x; h < total; h += (size_t)gridDim.x * blockDim.x) {
        const size_t idx = h * 2;
        const size_t x = idx & (N - 1);
        const size_t r = idx >> log_n;  // (b*2 + k)*nl + i
        const int i = (int)(r % nl);
        const size_t bk = r / nl;
        const int k = (int)(bk & 1);
        const size_t b = bk >> 1;
        const u64 q = __ldg(&tab->qq[i]), pinv = __ldg(&tab->pinv[i]), pinvsh = __ldg(&tab->pinv_sh[i]);
        const ulonglong2 vv = ld2(v + (bk * rows + i) * N + x);
        const ulonglong2 cc = ld2(conv + (bk * nl + i) * N + x);
        u64 o0 = mul_shoup(sub_mod(vv.x, cc.x, q), pinv, pinvsh, q);
        u64 o1 = mul_shoup(sub_mod(vv.y, cc.y, q), pinv, pinvsh, q);
        const u64* add = k == 0 ? add0 : add1;
        if (add) {
            const ulonglong2 aa = *reinterpret_cast<const ulonglong2*>(add + b * (k == 0 ? add0_stride : add1_stride) +
                                                                       ((size_t)i << log_n) + x);
            o0 = add_mod(o0, aa.x, q);
            o1 = add_mod(o1, aa.y, q);
        }
        st2(w + b * w_stride + ((size_t)(k * nl + i) << log_n) + x, o0, o1);
    }
}

// ---------------------------------------------------------------------------- ModDown + rescale
// A relinearisation followed by a rescale, fused so that each limb i < l of the result takes one
// forward NTT instead of two.  With x = add + (v - NTT(conv)) P^-1 the ModDown output and
// r = NTT([x_l]_{q_i}) the rescale's correction, NTT linearity gives exactly
//   (x_i - r_i) q_l^-1 = (add_i + v_i P^-1 - NTT(z_i)) q_l^-1,   z_i = conv_i P^-1 + [x_l]_{q_i},
// and the last limb x_l itself is formed in the coefficient domain from iNTT(add_l), iNTT(v_l)
// and conv_l.  Preparation: one thread per coefficient of one polynomial (bk = item * 2 + poly);
// v_l, the special-prime rows and al (= add_l) are in the coefficient domain; z overwrites conv.
__global__ void k_mdrs_prep(const u64* __restrict__ v, const u64* __restrict__ al, u64* __restrict__ conv, int B2,
                            int nl, int rows, int log_n, const ModDownTab* __restrict__ md,
                            const RescaleTab* __restrict__ rs, const ModConst* __restrict__ mc) {
    const size_t N = (size_t)1 << log_n;
    const size_t total = (size_t)B2 * N;
    const int L = nl - 1;
    const u64 ql = mc[L].q;
    const u64 pl = __ldg(&md->pinv[L]), pl_sh = __ldg(&md->pinv_sh[L]);
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
        const size_t x = idx & (N - 1), bk = idx >> log_n;
        u64* cb = conv + bk * nl * N + x;
        const u64 vl = v[(bk * rows + L) * N + x];
        const u64 xl = add_mod(mul_shoup(sub_mod(vl, cb[(size_t)L << log_n], ql), pl, pl_sh, ql), al[idx], ql);
        const bool neg = xl > (ql >> 1);
        for (int i = 0; i < L; i++) {
            const ModConst m = mc[i];
            u64 r = reduce64(xl, m);
            if (neg) r = add_mod(r, __ldg(&rs->negq[i]), m.q);
            const u64 cv = cb[(size_t)i << log_n];
            cb[(size_t)i << log_n] = add_mod(mul_shoup(cv, __ldg(&md->pinv[i]), __ldg(&md->pinv_sh[i]), m.q), r, m.q);
        }
    }
}

// out[b][k][i] = (add_k,i + v_k,i P^-1 - z_k,i) q_l^-1 for i < l (evaluation domain), 2
// coefficients per thread; grid-stride over B*2*l*N/2
__global__ void k_mdrs_combine(const u64* __restrict__ v, const u64* __restrict__ z, int B, int nl, int rows,
                               int log_n, const ModDownTab* __restrict__ md, const RescaleTab* __restrict__ rs,
                               const ModConst* __restrict__ mc, const u64* add0, size_t add0_stride,
                               const u64* add1, size_t add1_stride, u64* out, size_t out_stride) {
    const size_t N = (size_t)1 << log_n;
    const int L = nl - 1;
    const size_t total = (size_t)B * 2 * L * N / 2;
    for (size_t h = (size_t)blockIdx.x * blockDim.x + threadIdx.x; h < total; h += (size_t)gridDim.x * blockDim.x) {
        const size_t idx = h * 2;
        const size_t x = idx & (N - 1);
        const size_t r = idx >> log_n;  // (b*2 + k)*L + i
        const int i = (int)(r % L);
        const size_t bk = r / L;
        const int k = (int)(bk & 1);
        const size_t b = bk >> 1;
        const u64 q = mc[i].q;
        const u64 pinv = __ldg(&md->pinv[i]), pinvsh = __ldg(&md->pinv_sh[i]);
        const u64 qinv = __ldg(&rs->qinv[i]), qinvsh = __ldg(&rs->qinv_sh[i]);
        const ulonglong2 vv = ld2(v + (bk * rows + i) * N + x);
        const ulonglong2 zz = ld2(z + (bk * nl + i) * N + x);
        const u64* add = k == 0 ? add0 + b * add0_stride : add1 + b * add1_stride;
        const ulonglong2 aa = ld2(add + ((size_t)i << log_n) + x);
        const u64 o0 = mul_shoup(sub_mod(add_mod(aa.x, mul_shoup(vv.x, pinv, pinvsh, q), q), zz.x, q), qinv, qinvsh, q);
        const u64 o1 = mul_shoup(sub_mod(add_mod(aa.y, mul_shoup(vv.y, pinv, pinvsh, q), q), zz.y, q), qinv, qinvsh, q);
        st2(out + b * out_stride + ((size_t)(k * L + i) << log_n) + x, o0, o1);
    }
}

// ---------------------------------------------------------------------------- rescale
__global__ void k_rescale_prep(const u64* __restrict__ lastc, int Bdeg, int level, int log_n,
                               const RescaleTab* __restrict__ tab, const ModConst* __restrict__ mc,
                               u64* __restrict__ r) {
    const size_t N = (size_t)1 << log_n;
    const size_t total = (size_t)Bdeg * N;
    const u64 ql = mc[level].q;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
        const size_t x = idx & (N - 1), bd = idx >> log_n;
        const u64 v = lastc[idx];
        const bool neg = v > (ql >> 1);
        u64* rb = r + bd * level * N + x;
        for (int i = 0; i < level; i++) {
            const ModConst m = mc[i];
            u64 rv = reduce64(v, m);
            if (neg) rv = add_mod(rv, tab->negq[i], m.q);
            rb[(size_t)i << log_n] = rv;
        }
    }
}

__global__ void k_rescale_combine(const u64* __restrict__ ct, const u64* __restrict__ r, int B, int deg, int level,
                                  int log_n, const RescaleTab* __restrict__ tab, const ModConst* __restrict__ mc,
                                  u64* __restrict__ out) {
    const size_t N = (size_t)1 << log_n;
    const size_t total = (size_t)B * deg * level * N;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
        const size_t x = idx & (N - 1);
        const size_t rr = idx >> log_n;  // bd * level + i
        const int i = (int)(rr % level);
        const size_t bd = rr / level;
        const ModConst m = mc[i];
        const u64 xv = ct[(bd * (level + 1) + i) * N + x];
        out[idx] = mul_shoup(sub_mod(xv, r[idx], m.q), tab->qinv[i], tab->qinv_sh[i], m.q);
    }
}

// ---------------------------------------------------------------------------- automorphism
// y[p][r][idx] (+)= w[p][r][perm_g(idx)] over n_polys polys of `rows` rows; row r uses modulus
// r (r < nlq, a q row) or nq + r - nlq (a special-prime row)
__global__ void k_gather(const u64* __restrict__ w, u64* __restrict__ y, int n_polys, int rows, int nlq, int nq,
                         int log_n, uint64_t g, const ModConst* __restrict__ mc, int accumulate) {
    const size_t N = (size_t)1 << log_n;
    const size_t total = (size_t)n_polys * rows * N;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
        const unsigned x = (unsigned)(idx & (N - 1));
        const size_t row = idx >> log_n;
        const u64 val = w[(row << log_n) + auto_src(x, g, log_n)];
        if (accumulate) {
            const int r = (int)(row % rows);
            const u64 q = mc[r < nlq ? r : nq + (r - nlq)].q;
            y[idx] = add_mod(y[idx], val, q);
        } else {
            y[idx] = val;
        }
    }
}

// acc[b][i][idx] += src[b*src_stride + i*N + perm_g(idx)] for B items of nl q rows
__global__ void k_gather_items(const u64* __restrict__ src, size_t src_stride, u64* __restrict__ acc, int B, int nl,
                               int log_n, uint64_t g, const ModConst* __restrict__ mc) {
    const size_t N = (size_t)1 << log_n;
    const size_t total = (size_t)B * nl * N;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
        const unsigned x = (unsigned)(idx & (N - 1));
        const size_t row = idx >> log_n;
        const int i = (int)(row % nl);
        const size_t b = row / nl;
        const u64 val = src[b * src_stride + ((size_t)i << log_n) + auto_src(x, g, log_n)];
        acc[idx] = add_mod(acc[idx], val, mc[i].q);
    }
}

__global__ void k_permute_rows(const u64* __restrict__ in, u64* __restrict__ out, int rows, int log_n, uint64_t g) {
    const size_t N = (size_t)1 << log_n;
    const size_t total = (size_t)rows * N;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
        const unsigned x = (unsigned)(idx & (N - 1));
        const size_t row = idx >> log_n;
        out[idx] = in[(row << log_n) + auto_src(x, g, log_n)];
    }
}

// ---------------------------------------------------------------------------- keys / enc / dec
template <typename T>
__global__ void k_to_rns(const T* __restrict__ x, int B, ModList ml, int log_n, const ModConst* __restrict__ mc,
                         u64* __restrict__ out) {
    const size_t N = (size_t)1 << log_n;
    const size_t total = (size_t)B * ml.n * N;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
        const size_t c = idx & (N - 1);
        const size_t br = idx >> log_n;
        const int r = (int)(br % ml.n);
        const size_t b = br / ml.n;
        out[idx] = signed_to_res((int64_t)x[b * N + c], mc[ml.m[r]]);
    }
}

__global__ void k_key_combine(const u64* __restrict__ a, const u64* __restrict__ s, const u64* __restrict__ e,
                              const u64* __restrict__ st, ModList ml, int log_n, const ModConst* __restrict__ mc,
                              u64* __restrict__ b_out) {
    const size_t N = (size_t)1 << log_n;
    const size_t total = (size_t)ml.n * N;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(idx >> log_n);
        const ModConst m = mc[ml.m[r]];
        u64 v = sub_mod(e[idx], mul_mod(a[idx], s[idx], m), m.q);
        if (ml.flag[r]) v = add_mod(v, mul_mod(ml.val[r], st[idx], m), m.q);
        b_out[idx] = v;
    }
}

__global__ void k_enc_combine(const u64* __restrict__ mm, const u64* __restrict__ r, const u64* __restrict__ e0,
                              const u64* __restrict__ e1, const u64* __restrict__ pk, int B, int nl, int log_n,
                              const ModConst* __restrict__ mc, u64* __restrict__ out) {
    const size_t N = (size_t)1 << log_n;
    const size_t P = (size_t)nl * N;
    const size_t total = (size_t)B * P;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
        const size_t b = idx / P, o = idx - b * P;
        const ModConst m = mc[o >> log_n];
        const u64 rv = r[idx];
        const u64 c0 = add_mod(add_mod(mm[idx], mul_mod(rv, pk[o], m), m.q), e0[idx], m.q);
        const u64 c1 = add_mod(mul_mod(rv, pk[P + o], m), e1[idx], m.q);
        out[b * 2 * P + o] = c0;
        out[b * 2 * P + P + o] = c1;
    }
}

__global__ void k_dec_combine(const u64* __restrict__ ct, const u64* __restrict__ s, int deg, int nl, int log_n,
                              const ModConst* __restrict__ mc, u64* __restrict__ out) {
    const size_t N = (size_t)1 << log_n;
    const size_t P = (size_t)nl * N;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < P; idx += (size_t)gridDim.x * blockDim.x) {
        const ModConst m = mc[idx >> log_n];
        const u64 sv = s[idx];
        u64 acc = ct[idx], sp = sv;
        for (int p = 1; p < deg; p++) {
            acc = add_mod(acc, mul_mod(ct[(size_t)p * P + idx], sp, m), m.q);
            sp = mul_mod(sp, sv, m);
        }
        out[idx] = acc;
    }
}

__global__ void k_square_rows(const u64* __restrict__ s, u64* __restrict__ out, ModList ml, int log_n,
                              const ModConst* __restrict__ mc) {
    const size_t N = (size_t)1 << log_n;
    const size_t total = (size_t)ml.n * N;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
        const ModConst m = mc[ml.m[idx >> log_n]];
        out[idx] = mul_mod(s[idx], s[idx], m);
    }
}

unsigned grid_for(size_t total) {
    size_t g = (total + kT - 1) / kT;
    if (g > 148u * 64u) g = 148u * 64u;
    return (unsigned)(g ? g : 1);
}

}  // namespace

// ------------------------------------------------------------------------------------ launchers
void op_addsub(lc_ctx* c, const u64* a, const u64* b, u64* out, int n_polys, int nl, bool sub) {
    const size_t total = (size_t)n_polys * nl * c->N;
    k_addsub<<<grid_for(total), kT, 0, c->stream>>>(a, b, out, nl, c->log_n, total, c->mc, sub ? 1 : 0);
    g_lc_launches += 1;
}

void op_tensor(lc_ctx* c, const u64* a, const u64* b, u64* out, int nl) {
    const size_t P = (size_t)nl * c->N;
    k_tensor<<<grid_for(P), kT, 0, c->stream>>>(a, b, out, c->log_n, P, c->mc);
    g_lc_launches += 1;
}

void op_sq_acc_pairs(lc_ctx* c, const u64* cts, int n, int chunks, int nl, int p0, int np, u64* out) {
    dim3 grid(np, (unsigned)(c->N / kT), nl);
    k_sq_acc_pairs<<<grid, kT, 0, c->stream>>>(cts, n, chunks, nl, c->log_n, p0, c->mc, out);
    g_lc_launches += 1;
}

// the tensor kernels' ring lives in dynamic shared memory (above the 48 KB static limit); the
// attribute is set once per kernel instantiation
template <typename K>
static void tensor_smem_attr(K kernel) {
    static std::mutex mu;
    static std::set<const void*> done;  // kernels whose attribute is set
    std::lock_guard<std::mutex> lock(mu);
    if (done.insert(reinterpret_cast<const void*>(kernel)).second)
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTensorSmem);
}

// first limb of the range [split0, nl) whose primes are all below 2^40 (20-bit split products)
static int split_start(lc_ctx* c, int nl) {
    int s0 = nl;
    while (s0 > 0 && c->mod[s0 - 1] < (1ull << 40)) s0--;
    return s0;
}

void op_sq_acc_tiled(lc_ctx* c, const u64* cts, int n, int chunks, int nl, int p0, int np, u64* out) {
    const int cb = n <= 11 ? n : 8;  // one diagonal block up to 11 clients (55 pairs), else blocks of 8
    const int nb = (n + cb - 1) / cb;
    // limbs [split0, nl) take the 20-bit split path (partial sums stay below 2^64 for < 2^20 chunks)
    int split0 = split_start(c, nl);
    if (chunks > (1 << 20)) split0 = nl;
    if (split0 > 0) {
        dim3 grid(nb * (nb + 1) / 2, (unsigned)(c->N / kTX), split0);
        tensor_smem_attr(k_sq_acc_tiled<16, 4, false>);
        k_sq_acc_tiled<16, 4, false><<<grid, 512, kTensorSmem, c->stream>>>(cts, n, chunks, nl, 0, c->log_n, cb, p0,
                                                                             np, c->mc, out);
        g_lc_launches += 1;
    }
    if (split0 < nl) {  // warps per block: LC_TUNE_TENSOR_WARPS (pair slots per thread = 64 / warps, rounded up)
        dim3 grid(nb * (nb + 1) / 2, (unsigned)(c->N / kTX), nl - split0);
        switch (c->tune[LC_TUNE_TENSOR_WARPS]) {
            case 8:
                tensor_smem_attr(k_sq_acc_tiled<8, 8, true>);
                k_sq_acc_tiled<8, 8, true><<<grid, 256, kTensorSmem, c->stream>>>(cts, n, chunks, nl, split0, c->log_n,
                                                                                   cb, p0, np, c->mc, out);
                break;
            case 12:
                tensor_smem_attr(k_sq_acc_tiled<12, 6, true>);
                k_sq_acc_tiled<12, 6, true><<<grid, 384, kTensorSmem, c->stream>>>(cts, n, chunks, nl, split0,
                                                                                    c->log_n, cb, p0, np, c->mc, out);
                break;
            default:
                tensor_smem_attr(k_sq_acc_tiled<16, 4, true>);
                k_sq_acc_tiled<16, 4, true><<<grid, 512, kTensorSmem, c->stream>>>(cts, n, chunks, nl, split0,
                                                                                    c->log_n, cb, p0, np, c->mc, out);
                break;
        }
        g_lc_launches += 1;
    }
}

void op_mask_acc(lc_ctx* c, const u64* cts, int n, int chunks, int nl, const u64* masks, int k0, int nk, u64* out) {
    // limbs [split0, nl): 20-bit split products (sum (h l' + l h') of n clients stays below 2^64
    // for n < 2^21)
    int split0 = split_start(c, nl);
    if (n >= (1 << 21)) split0 = nl;
    if (split0 > 0) {
        dim3 grid(nk, (unsigned)(c->N / kT), split0);
        k_mask_acc<false><<<grid, kT, 0, c->stream>>>(cts, n, chunks, nl, 0, c->log_n, k0, masks, c->mc, out);
        g_lc_launches += 1;
    }
    if (split0 < nl) {
        dim3 grid(nk, (unsigned)(c->N / kT), nl - split0);
        k_mask_acc<true><<<grid, kT, 0, c->stream>>>(cts, n, chunks, nl, split0, c->log_n, k0, masks, c->mc, out);
        g_lc_launches += 1;
    }
}

void op_modup(lc_ctx* c, const u64* coef, size_t coef_stride, int B, int level, u64* ext) {
    const int beta = c->digits(level);
    const int rows = level + 1 + c->np;
    const int nl = level + 1;
    const ModUpTab* tabs = c->modup + (size_t)level * c->dnum;
    // digits 0..beta-2 have alpha primes; the last one has the remainder
    const int last = nl - (beta - 1) * c->alpha;
    auto launch = [&](int ns, int j0, int nj) {
        dim3 grid((unsigned)(c->N / (2 * kT)), B * nj);
        switch (ns) {
            case 1: k_modup<1><<<grid, kT, 0, c->stream>>>(coef, coef_stride, beta, j0, nj, rows, c->log_n, tabs, ext); break;
            case 2: k_modup<2><<<grid, kT, 0, c->stream>>>(coef, coef_stride, beta, j0, nj, rows, c->log_n, tabs, ext); break;
            case 3: k_modup<3><<<grid, kT, 0, c->stream>>>(coef, coef_stride, beta, j0, nj, rows, c->log_n, tabs, ext); break;
            case 4: k_modup<4><<<grid, kT, 0, c->stream>>>(coef, coef_stride, beta, j0, nj, rows, c->log_n, tabs, ext); break;
            case 5: k_modup<5><<<grid, kT, 0, c->stream>>>(coef, coef_stride, beta, j0, nj, rows, c->log_n, tabs, ext); break;
            case 6: k_modup<6><<<grid, kT, 0, c->stream>>>(coef, coef_stride, beta, j0, nj, rows, c->log_n, tabs, ext); break;
            case 7: k_modup<7><<<grid, kT, 0, c->stream>>>(coef, coef_stride, beta, j0, nj, rows, c->log_n, tabs, ext); break;
            case 8: k_modup<8><<<grid, kT, 0, c->stream>>>(coef, coef_stride, beta, j0, nj, rows, c->log_n, tabs, ext); break;
            default: break;
        }
        g_lc_launches += 1;
    };
    if (last == c->alpha) {
        launch(c->alpha, 0, beta);
    } else {
        if (beta > 1) launch(c->alpha, 0, beta - 1);
        launch(last, beta - 1, 1);
    }
}

void op_inner(lc_ctx* c, const u64* ext, const u64* d, size_t d_stride, int B, int level, const u64* key, u64* v) {
    const int beta = c->digits(level);
    const int nl = level + 1, rows = nl + c->np;
    dim3 grid(B, (unsigned)(c->N / (4 * kT)), rows);
    k_inner<<<grid, kT, 0, c->stream>>>(ext, d, d_stride, beta, nl, rows, c->alpha, c->nq, c->nq + c->np, c->log_n,
                                        key, c->mc, v);
    g_lc_launches += 1;
}

void op_inner_multi(lc_ctx* c, const u64* ext, const u64* d, size_t d_stride, int B, int level, const u64* const* keys,
                    int T, u64* v, size_t v_key_stride) {
    const int beta = c->digits(level);
    const int nl = level + 1, rows = nl + c->np;
    dim3 grid(B, (unsigned)(c->N / (2 * kT)), rows);
    KeyPtrs kp{};
    for (int k = 0; k < T && k < 8; k++) kp.p[k] = keys[k];
#define LC_IM(TT)                                                                                                   \
    k_inner_multi<TT><<<grid, kT, 0, c->stream>>>(ext, d, d_stride, beta, nl, rows, c->alpha, c->nq, c->nq + c->np, \
                                                  c->log_n, kp, c->mc, v, v_key_stride)
    switch (T) {
        case 1: LC_IM(1); break;
        case 2: LC_IM(2); break;
        case 3: LC_IM(3); break;
        case 4: LC_IM(4); break;
        case 5: LC_IM(5); break;
        case 6: LC_IM(6); break;
        case 7: LC_IM(7); break;
        default: break;
    }
#undef LC_IM
    g_lc_launches += 1;
}

void op_inner_gather(lc_ctx* c, const u64* ext, const u64* d, size_t d_stride, const u64* y0, size_t y0_stride, int B,
                     int level, const u64* const* keys, const u64* const* keys_dev, const uint64_t* gs, int T,
                     u64* usum, u64* c0acc) {
    const int beta = c->digits(level);
    const int nl = level + 1, rows = nl + c->np;
    KeyPtrs kp{};
    Galois g{};
    for (int k = 0; k < T && k < 16; k++) {
        kp.p[k] = keys ? keys[k] : nullptr;
        g.g[k] = gs[k];
    }
    // Q rows [k, nl) whose primes are all below 2^40 take the split-product kernel; rows [0, k)
    // and the special primes take the 128-bit one
    int k = nl;
    while (k > 0 && c->mod[k - 1] < (1ull << 40)) k--;
    const RowSel split{k, nl - k, 0}, wide{0, k, nl};
    const int ns = nl - k, nw = k + c->np;
    const unsigned gy = (unsigned)(c->N / (2 * kTG));
#define LC_IG(TT, SPL, BT, SEL, CNT, KA)                                                                            \
    {                                                                                                               \
        const dim3 grid((unsigned)((B + BT - 1) / BT), gy, CNT);                                                    \
        if (keys_dev)                                                                                               \
            k_inner_gather<TT, true, SPL, BT, KA><<<grid, kTG, 0, c->stream>>>(                                     \
                ext, d, d_stride, y0, y0_stride, B, beta, nl, rows, c->alpha, c->nq, c->nq + c->np, c->log_n, kp,    \
                keys_dev, g, SEL, c->mc, usum, c0acc);                                                              \
        else                                                                                                        \
            k_inner_gather<TT, false, SPL, BT, KA><<<grid, kTG, 0, c->stream>>>(                                    \
                ext, d, d_stride, y0, y0_stride, B, beta, nl, rows, c->alpha, c->nq, c->nq + c->np, c->log_n, kp,    \
                nullptr, g, SEL, c->mc, usum, c0acc);                                                               \
    }
    // groups of 2, 3 and 4 rotation bits (a group of one rotation takes the per-rotation path)
#define LC_IG_T(SPL, BT, SEL, CNT, KA)                  \
    switch (T) {                                        \
        case 3: LC_IG(3, SPL, BT, SEL, CNT, KA); break;   \
        case 7: LC_IG(7, SPL, BT, SEL, CNT, KA); break;   \
        case 15: LC_IG(15, SPL, BT, SEL, CNT, KA); break; \
        default: break;                                 \
    }
    if (ns) {  // items per thread: LC_TUNE_GROUP_SPLIT_ITEMS; products: LC_TUNE_GROUP_KARATSUBA
        const bool kara = c->tune[LC_TUNE_GROUP_KARATSUBA] == 1;
        if (c->tune[LC_TUNE_GROUP_SPLIT_ITEMS] == 2) {
            if (kara) LC_IG_T(true, 2, split, ns, true) else LC_IG_T(true, 2, split, ns, false)
        } else {
            if (kara) LC_IG_T(true, 1, split, ns, true) else LC_IG_T(true, 1, split, ns, false)
        }
        g_lc_launches += 1;
    }
    if (nw) {  // LC_TUNE_GROUP_WIDE_ITEMS
        if (c->tune[LC_TUNE_GROUP_WIDE_ITEMS] == 1) {
            LC_IG_T(false, 1, wide, nw, false)
        } else {
            LC_IG_T(false, 2, wide, nw, false)
        }
        g_lc_launches += 1;
    }
#undef LC_IG_T
#undef LC_IG
}

void op_gather_sum_qp(lc_ctx* c, const u64* src, size_t src_stride, u64* usum, int n_polys, int nl,
                      const uint64_t* gs, int T) {
    const int rows = nl + c->np;
    const size_t total = (size_t)n_polys * rows * c->N;
    Galois g{};
    for (int k = 0; k < T && k < 8; k++) g.g[k] = gs[k];
#define LC_GS(TT)                                                                                                \
    k_gather_sum<TT><<<grid_for(total), kT, 0, c->stream>>>(src, src_stride, usum, n_polys, rows, nl, c->nq, c->log_n, \
                                                            g, c->mc)
    switch (T) {
        case 1: LC_GS(1); break;
        case 2: LC_GS(2); break;
        case 3: LC_GS(3); break;
        case 4: LC_GS(4); break;
        case 5: LC_GS(5); break;
        case 6: LC_GS(6); break;
        case 7: LC_GS(7); break;
        default: break;
    }
#undef LC_GS
    g_lc_launches += 1;
}

void op_moddown_bconv(lc_ctx* c, const u64* v, int B, int level, u64* conv) {
    const int nl = level + 1, rows = nl + c->np;
    dim3 grid((unsigned)(c->N / (2 * kT)), B * 2);
    switch (c->np) {
        case 1: k_moddown_bconv<1><<<grid, kT, 0, c->stream>>>(v, nl, rows, c->log_n, c->moddown, conv); break;
        case 2: k_moddown_bconv<2><<<grid, kT, 0, c->stream>>>(v, nl, rows, c->log_n, c->moddown, conv); break;
        case 3: k_moddown_bconv<3><<<grid, kT, 0, c->stream>>>(v, nl, rows, c->log_n, c->moddown, conv); break;
        case 4: k_moddown_bconv<4><<<grid, kT, 0, c->stream>>>(v, nl, rows, c->log_n, c->moddown, conv); break;
        case 5: k_moddown_bconv<5><<<grid, kT, 0, c->stream>>>(v, nl, rows, c->log_n, c->moddown, conv); break;
        case 6: k_moddown_bconv<6><<<grid, kT, 0, c->stream>>>(v, nl, rows, c->log_n, c->moddown, conv); break;
        case 7: k_moddown_bconv<7><<<grid, kT, 0, c->stream>>>(v, nl, rows, c->log_n, c->moddown, conv); break;
        case 8: k_moddown_bconv<8><<<grid, kT, 0, c->stream>>>(v, nl, rows, c->log_n, c->moddown, conv); break;
        default: break;
    }
    g_lc_launches += 1;
}

void op_moddown_combine(lc_ctx* c, const u64* v, const u64* conv, int B, int level, const u64* add0,
                        size_t add0_stride, const u64* add1, size_t add1_stride, u64* w, size_t w_stride) {
    const int nl = level + 1, rows = nl + c->np;
    const size_t total = (size_t)B * 2 * nl * c->N / 2;
    k_moddown_combine<<<grid_for(total), kT, 0, c->stream>>>(v, conv, B, nl, rows, c->log_n, c->moddown, c->mc, add0,
                                                             add0_stride, add1, add1_stride, w, w_stride);
    g_lc_launches += 1;
}

void op_mdrs_prep(lc_ctx* c, const u64* v, const u64* al, u64* conv, int B, int level) {
    const int nl = level + 1, rows = nl + c->np;
    const size_t total = (size_t)B * 2 * c->N;
    k_mdrs_prep<<<grid_for(total), kT, 0, c->stream>>>(v, al, conv, B * 2, nl, rows, c->log_n, c->moddown,
                                                       c->rescale + level, c->mc);
    g_lc_launches += 1;
}

void op_mdrs_combine(lc_ctx* c, const u64* v, const u64* z, int B, int level, const u64* add0, size_t add0_stride,
                     const u64* add1, size_t add1_stride, u64* out, size_t out_stride) {
    const int nl = level + 1, rows = nl + c->np;
    const size_t total = (size_t)B * 2 * level * c->N / 2;
    k_mdrs_combine<<<grid_for(total), kT, 0, c->stream>>>(v, z, B, nl, rows, c->log_n, c->moddown, c->rescale + level,
                                                          c->mc, add0, add0_stride, add1, add1_stride, out,
                                                          out_stride);
    g_lc_launches += 1;
}

void op_rescale_prep(lc_ctx* c, const u64* lastc, int Bdeg, int level, u64* r) {
    const size_t total = (size_t)Bdeg * c->N;
    k_rescale_prep<<<grid_for(total), kT, 0, c->stream>>>(lastc, Bdeg, level, c->log_n, c->rescale + level, c->mc, r);
    g_lc_launches += 1;
}

void op_rescale_combine(lc_ctx* c, const u64* ct, const u64* r, int B, int deg, int level, u64* out) {
    const size_t total = (size_t)B * deg * level * c->N;
    k_rescale_combine<<<grid_for(total), kT, 0, c->stream>>>(ct, r, B, deg, level, c->log_n, c->rescale + level, c->mc,
                                                             out);
    g_lc_launches += 1;
}

void op_gather(lc_ctx* c, const u64* w, u64* y, int n_polys, int nl, uint64_t g, bool accumulate) {
    const size_t total = (size_t)n_polys * nl * c->N;
    k_gather<<<grid_for(total), kT, 0, c->stream>>>(w, y, n_polys, nl, nl, c->nq, c->log_n, g, c->mc,
                                                    accumulate ? 1 : 0);
    g_lc_launches += 1;
}

void op_gather_c0(lc_ctx* c, const u64* ct, u64* acc, int B, int nl, uint64_t g) {
    const size_t total = (size_t)B * nl * c->N;
    k_gather_items<<<grid_for(total), kT, 0, c->stream>>>(ct, (size_t)2 * nl * c->N, acc, B, nl, c->log_n, g, c->mc);
    g_lc_launches += 1;
}

void op_gather_qp(lc_ctx* c, const u64* w, u64* y, int n_polys, int nl, uint64_t g, bool accumulate) {
    const int rows = nl + c->np;
    const size_t total = (size_t)n_polys * rows * c->N;
    k_gather<<<grid_for(total), kT, 0, c->stream>>>(w, y, n_polys, rows, nl, c->nq, c->log_n, g, c->mc,
                                                    accumulate ? 1 : 0);
    g_lc_launches += 1;
}

void op_permute_rows(lc_ctx* c, const u64* in, u64* out, int rows, uint64_t g) {
    const size_t total = (size_t)rows * c->N;
    k_permute_rows<<<grid_for(total), kT, 0, c->stream>>>(in, out, rows, c->log_n, g);
    g_lc_launches += 1;
}

void op_to_rns_i64(lc_ctx* c, const int64_t* x, int B, const int* mods, int nrows, u64* out) {
    ModList ml = make_list(mods, nrows);
    k_to_rns<int64_t><<<grid_for((size_t)B * nrows * c->N), kT, 0, c->stream>>>(x, B, ml, c->log_n, c->mc, out);
    g_lc_launches += 1;
}
void op_to_rns_i32(lc_ctx* c, const int32_t* x, int B, const int* mods, int nrows, u64* out) {
    ModList ml = make_list(mods, nrows);
    k_to_rns<int32_t><<<grid_for((size_t)B * nrows * c->N), kT, 0, c->stream>>>(x, B, ml, c->log_n, c->mc, out);
    g_lc_launches += 1;
}
void op_to_rns_i8(lc_ctx* c, const int8_t* x, int B, const int* mods, int nrows, u64* out) {
    ModList ml = make_list(mods, nrows);
    k_to_rns<int8_t><<<grid_for((size_t)B * nrows * c->N), kT, 0, c->stream>>>(x, B, ml, c->log_n, c->mc, out);
    g_lc_launches += 1;
}

void op_key_combine(lc_ctx* c, const u64* a, const u64* s, const u64* e, const u64* st, const u64* addmul,
                    const int* mods, int nrows, u64* b_out) {
    ModList ml = make_list(mods, nrows, addmul);
    k_key_combine<<<grid_for((size_t)nrows * c->N), kT, 0, c->stream>>>(a, s, e, st, ml, c->log_n, c->mc, b_out);
    g_lc_launches += 1;
}

void op_enc_combine(lc_ctx* c, const u64* m, const u64* r, const u64* e0, const u64* e1, const u64* pk, int B, int nl,
                    u64* out) {
    k_enc_combine<<<grid_for((size_t)B * nl * c->N), kT, 0, c->stream>>>(m, r, e0, e1, pk, B, nl, c->log_n, c->mc,
                                                                         out);
    g_lc_launches += 1;
}

void op_dec_combine(lc_ctx* c, const u64* ct, const u64* s, int deg, int nl, u64* out) {
    k_dec_combine<<<grid_for((size_t)nl * c->N), kT, 0, c->stream>>>(ct, s, deg, nl, c->log_n, c->mc, out);
    g_lc_launches += 1;
}

void op_square_rows(lc_ctx* c, const u64* s, u64* out, const int* mods, int nrows) {
    ModList ml = make_list(mods, nrows);
    k_square_rows<<<grid_for((size_t)nrows * c->N), kT, 0, c->stream>>>(s, out, ml, c->log_n, c->mc);
    g_lc_launches += 1;
}

void op_readout_finish(lc_ctx* c, const u64* res, int count, double scale, double* out) {
    if (count <= 0) return;
    k_readout_finish<<<(count + kT - 1) / kT, kT, 0, c->stream>>>(res, count, c->mc, scale, out);
    g_lc_launches += 1;
}

void op_krum(lc_ctx* c, const double* d, int n, int f, int l, int average, double* w, int* sel) {
    k_krum<<<1, 256, 0, c->stream>>>(d, n, f, l, average, w, sel);
    g_lc_launches += 1;
}

// encode `count` slot vectors z [count][N/2] (device doubles) into m [count][N] (device int64);
// A = scratch of count * 2N double2; tables: pos [N/2], w256 [256], wbig [2N]
void op_encode(lc_ctx* c, const double* z, int count, double scale, const unsigned* pos, const double2* w256,
               const double2* wbig, double2* A, int64_t* m) {
    if (count <= 0) return;
    const size_t N = c->N;
    cudaMemsetAsync(A, 0, (size_t)count * 2 * N * sizeof(double2), c->stream);
    k_enc_scatter<<<grid_for((size_t)count * N / 2), kT, 0, c->stream>>>(z, count, c->log_n, pos, scale, A);
    const int log_2n = c->log_n + 1;
    k_fft_cols<<<dim3((unsigned)((2 * N >> 8) / 8), count), 128, 0, c->stream>>>(A, log_2n, w256, wbig);
    k_fft_rows_out<<<dim3(256 / 8, count), 128, 0, c->stream>>>(A, c->log_n, w256, m);
    g_lc_launches += 3;
}

void op_pack_key(lc_ctx* c, const u64* in, u64* out, size_t words) {
    k_pack_key<<<grid_for(words), kT, 0, c->stream>>>(in, out, c->nq + c->np, c->log_n, c->mc, words);
    g_lc_launches += 1;
}

void op_sample_enc(lc_ctx* c, u64 seed, u64 first, int count, int8_t* r, int32_t* e0, int32_t* e1) {
    if (count <= 0) return;
    k_sample_enc<<<grid_for((size_t)count * c->N), kT, 0, c->stream>>>(seed, first, count, c->log_n, r, e0, e1);
    g_lc_launches += 1;
}

void op_const_plain(lc_ctx* c, const double* w, int count, double scale, int64_t* m) {
    if (count <= 0) return;
    k_const_plain<<<grid_for((size_t)count * c->N), kT, 0, c->stream>>>(w, count, c->log_n, scale, m);
    g_lc_launches += 1;
}

void op_mask_acc_items(lc_ctx* c, const AggItem* items_dev, int count, int nl, u64* out) {
    if (count <= 0) return;
    const int s0 = split_start(c, nl);  // a job's clients (< 2^21) fit the 64-bit partial sums
    if (s0 > 0) {
        dim3 grid(count, (unsigned)(c->N / kT), s0);
        k_mask_acc_items<false><<<grid, kT, 0, c->stream>>>(items_dev, nl, 0, c->log_n, c->mc, out);
        g_lc_launches += 1;
    }
    if (s0 < nl) {
        dim3 grid(count, (unsigned)(c->N / kT), nl - s0);
        k_mask_acc_items<true><<<grid, kT, 0, c->stream>>>(items_dev, nl, s0, c->log_n, c->mc, out);
        g_lc_launches += 1;
    }
}

void op_inner_items(lc_ctx* c, const u64* ext, const u64* d, size_t d_stride, int B, int level,
                    const u64* const* keys_dev, int T, u64* v, size_t v_key_stride) {
    const int beta = c->digits(level);
    const int nl = level + 1, rows = nl + c->np;
    dim3 grid(B, (unsigned)(c->N / (2 * kT)), rows);
#define LC_II(TT)                                                                                                   \
    k_inner_items<TT><<<grid, kT, 0, c->stream>>>(ext, d, d_stride, beta, nl, rows, c->alpha, c->nq, c->nq + c->np, \
                                                  c->log_n, keys_dev, c->mc, v, v_key_stride)
    switch (T) {
        case 1: LC_II(1); break;
        case 2: LC_II(2); break;
        case 3: LC_II(3); break;
        case 4: LC_II(4); break;
        case 5: LC_II(5); break;
        case 6: LC_II(6); break;
        case 7: LC_II(7); break;
        default: break;
    }
#undef LC_II
    g_lc_launches += 1;
}

void op_copy_items(lc_ctx* c, const u64* src, size_t words, u64* const* dst_dev, int B) {
    if (B <= 0) return;
    dim3 grid((unsigned)std::min<size_t>((words / 2 + kT - 1) / kT, 4096), B);
    k_copy_items<<<grid, kT, 0, c->stream>>>(src, words, dst_dev);
    g_lc_launches += 1;
}

void op_const_coef0(lc_ctx* c, const u64* cts, size_t ct_stride, int count, const u64* s0, u64* out) {
    if (count <= 0) return;
    k_const_coef0<<<count, kT, 0, c->stream>>>(cts, ct_stride, s0, c->log_n, c->mc, out);
    g_lc_launches += 1;
}


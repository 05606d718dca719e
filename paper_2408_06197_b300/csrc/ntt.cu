// Negacyclic NTT kernels; see ntt.cuh for the domain convention and pass structure.
//
// Column pass (index bits [8, log_n), C = log_n - 8 "row" bits of a 2^C x 256 view): a CTA of
// 2^C threads owns 16 columns; every thread loads 16 words straight from global memory (a warp
// reads two full 128-byte row segments per load), runs the top 4 row-bit stages in registers,
// exchanges once through shared memory, runs the remaining C-4 stages, and stores straight to
// global memory.  Row pass (bits [0, 8)): a CTA of 128 threads owns 8 blocks of 256 words; the
// two radix-16 halves are separated by one swizzled shared-memory exchange, and a second
// exchange restores a coalesced store (forward) or load (inverse).
#include <cuda_runtime.h>
#include <algorithm>
#include <map>
#include <mutex>
#include <utility>
#include "ntt.cuh"
#include "context.cuh"
#include "tma.cuh"
#include "probe.cuh"

namespace {

constexpr int kRowThreads = 128;

__device__ __forceinline__ u64* limb_ptr(u64* base, size_t batch_stride, const RowMap& map, int b, int log_n,
                                         int& mod_idx) {
    const int n = map.n;
    const int bi = b / n, r = b - bi * n;
    mod_idx = map.mod[r];
    return base + (size_t)bi * batch_stride + ((size_t)map.row[r] << log_n);
}

// Two value-range disciplines, chosen per CTA from the limb's prime:
//  * q >= 2^46 (the 50/60-bit primes): Harvey-lazy, forward values in [0, 4q) and inverse values in
//    [0, 2q), one conditional subtraction per butterfly;
//  * q < 2^46 (the 30/40-bit primes): no conditional subtraction inside the network, and the
//    products take the three-partial-product quotient of mul_shoup_lazy4 (results in [0, 4q)).
//    Forward values grow by less than 4q per stage (below 4q + 4q log2(N) <= 68q for inputs below
//    4q and log2(N) <= 16, inside the range reduce_lazy takes); inverse values start below 2q and
//    at most double per stage (below 2^(s+1) q after s >= 1 stages: each sum adds two such values,
//    each product is below 4q), so the multiple 2^(b+1) q used at stage b is never below the
//    subtracted value; the last stage reduces fully.  Outputs are the same canonical residues in
//    both disciplines.
constexpr u64 kLazyLimit = 1ull << 46;

// y w mod q up to 4q for any y < 2^64: the Shoup quotient floor(y w' / 2^64) from three of the
// four 32-bit partial products of y w' -- the low x low product and the carry out of the sum of
// the two middle products' low halves are left out, each of which moves the quotient by at most
// one -- so the estimate is the exact quotient or up to two below it, and y w - t q, in [0, 2q)
// with the exact one, lies in [0, 4q).
// The estimate is y1 w'1 + hi32(y0 w'1) + hi32(y1 w'0) (two high-half products, their 33-bit sum
// and one 32x32 -> 64-bit multiply-add), the remainder the chain of mul_sub_lo.
__device__ __forceinline__ u64 mul_shoup_lazy4(u64 y, u64 w, u64 w_sh, u64 q) {
    u64 t;
    asm("{\n\t"
        ".reg .u32 y0, y1, p0, p1, h1, h2, s0, s1;\n\t"
        ".reg .u64 s;\n\t"
        "mov.b64 {y0, y1}, %1;\n\t"
        "mov.b64 {p0, p1}, %2;\n\t"
        "mul.hi.u32 h1, y0, p1;\n\t"
        "mul.hi.u32 h2, y1, p0;\n\t"
        "add.cc.u32 s0, h1, h2;\n\t"
        "addc.u32 s1, 0, 0;\n\t"
        "mov.b64 s, {s0, s1};\n\t"
        "mad.wide.u32 %0, y1, p1, s;\n\t"
        "}"
        : "=l"(t)
        : "l"(y), "l"(w_sh));
    return mul_sub_lo(y, w, t, 0 - q);
}

// Cooley-Tukey butterfly; t = y w is in [0, 4q) (LZ) or [0, 2q) (exact lazy Shoup) for any y
template <bool LZ>
__device__ __forceinline__ void ct_bfly(u64& x, u64& y, ulonglong2 w, u64 q, u64 two_q) {
    const u64 xr = LZ ? x : csub(x, two_q);
    const u64 t = LZ ? mul_shoup_lazy4(y, w.x, w.y, q) : mul_shoup_lazy(y, w.x, w.y, q);
    x = xr + t;
    y = xr + (LZ ? two_q << 1 : two_q) - t;
}
// Gentleman-Sande butterfly; ky is a multiple of q not below y (LZ), else y < 2q
template <bool LZ>
__device__ __forceinline__ void gs_bfly(u64& x, u64& y, ulonglong2 w, u64 q, u64 two_q, u64 ky) {
    const u64 a = x + y;
    const u64 b = x + (LZ ? ky : two_q) - y;
    x = LZ ? a : csub(a, two_q);
    y = LZ ? mul_shoup_lazy4(b, w.x, w.y, q) : mul_shoup_lazy(b, w.x, w.y, q);
}

// swizzle for the row-pass tile: XOR word bits 0..3 with bits 4..7
__device__ __forceinline__ int swz(int e) { return e ^ ((e >> 4) & 15); }

__device__ __forceinline__ ulonglong2 ldtw(const ulonglong2* t, int i) { return __ldg(t + i); }

// Slot of the twiddle of the row-pass stages b = 0..3 that pair word g0 + 16 lo + u with its
// partner (g0 a multiple of 256, lo < 16, u < 16): logically entry 2^(log_n-1-b) +
// ((g0 + 16 lo + u) >> (b+1)).  The tables store each group of 16 * 2^(3-b) consecutive entries of
// the stages b = 0..2 lane-interleaved (entry lo * 2^(3-b) + v of a group at v * 16 + lo, see
// the table build), so that for one u the 16 lanes of a half-warp read 16 consecutive entries;
// for b = 3 the two orders coincide.
__device__ __forceinline__ int tw_row_slot(int log_n, int b, int g0, int lo, int u) {
    return (1 << (log_n - 1 - b)) + (g0 >> (b + 1)) + ((u >> (b + 1)) << 4) + lo;
}

// ------------------------------------------------------------------------------ column pass
// forward: row bits C-1 .. 0 (global bits log_n-1 .. 8)
template <int C, bool LZ>
__device__ __forceinline__ void fwd_col_body(u64* a, u64* s, const ModConst& mc, const ulonglong2* tw, int col0) {
    constexpr int LOGN = C + 8;
    constexpr int T = 1 << C;
    constexpr int RS = 1 << (C - 4);  // row stride of a thread's 16 words in phase 1
    constexpr int R2 = C - 4;         // row bits left for phase 2
    const int tid = threadIdx.x;
    const int c = tid & 15, rg = tid >> 4;
    u64 x[16];
#pragma unroll
    for (int u = 0; u < 16; u++) x[u] = a[((size_t)(rg + RS * u) << 8) + col0 + c];
#pragma unroll
    for (int st = 3; st >= 0; st--) {
        const int b = R2 + st;
#pragma unroll
        for (int u = 0; u < 16; u++) {
            if (u >> st & 1) continue;
            // row = rg + RS*u with rg < RS <= 2^b: row >> (b+1) = u >> (b+1-R2), a compile-time offset
            ct_bfly<LZ>(x[u], x[u | (1 << st)], ldtw(tw, (1 << (LOGN - 9 - b)) + (u >> (b + 1 - R2))), mc.q,
                        mc.two_q);
        }
    }
    if constexpr (R2 == 0) {
#pragma unroll
        for (int u = 0; u < 16; u++) a[((size_t)(rg + RS * u) << 8) + col0 + c] = x[u];
    } else {
#pragma unroll
        for (int u = 0; u < 16; u++) s[((rg + RS * u) << 4) + c] = x[u];
        __syncthreads();
        constexpr int V = 1 << R2;
#pragma unroll
        for (int k = 0; k < (256 >> C); k++) {
            const int item = tid + T * k;
            const int c2 = item & 15, grp = item >> 4;
            u64 y[V];
#pragma unroll
            for (int v = 0; v < V; v++) y[v] = s[(((grp << R2) + v) << 4) + c2];
#pragma unroll
            for (int st = R2 - 1; st >= 0; st--) {
                const int b = st;
#pragma unroll
                for (int v = 0; v < V; v++) {
                    if (v >> st & 1) continue;
                    ct_bfly<LZ>(y[v], y[v | (1 << st)],
                                ldtw(tw, (1 << (LOGN - 9 - b)) + ((grp << R2) >> (b + 1)) + (v >> (b + 1))), mc.q,
                                mc.two_q);
                }
            }
#pragma unroll
            for (int v = 0; v < V; v++) a[((size_t)((grp << R2) + v) << 8) + col0 + c2] = y[v];
        }
    }
}

template <int C, int MINB>
__global__ void __launch_bounds__(1 << C, MINB) ntt_fwd_col(u64* base, size_t batch_stride, RowMap map, NttTables tb) {
    constexpr int LOGN = C + 8;
    __shared__ u64 s[C > 4 ? (16 << C) : 1];
    int mi;
    u64* a = limb_ptr(base, batch_stride, map, blockIdx.y, LOGN, mi);
    const ModConst mc = tb.mc[mi];
    const ulonglong2* tw = tb.fwd + ((size_t)mi << LOGN);
    if (mc.q < kLazyLimit)
        fwd_col_body<C, true>(a, s, mc, tw, blockIdx.x * 16);
    else
        fwd_col_body<C, false>(a, s, mc, tw, blockIdx.x * 16);
}

// inverse: row bits 0 .. C-1 (global stages 8 .. log_n-1); the last stage (t = N/2) folds N^-1
template <int C, bool LZ>
__device__ __forceinline__ void inv_col_body(u64* a, u64* s, const ModConst& mc, const ulonglong2* tw, int col0) {
    constexpr int LOGN = C + 8;
    constexpr int T = 1 << C;
    constexpr int RS = 1 << (C - 4);
    constexpr int R2 = C - 4;
    const int tid = threadIdx.x;
    const int c = tid & 15, rg = tid >> 4;
    u64 x[16];
    if constexpr (R2 == 0) {
#pragma unroll
        for (int u = 0; u < 16; u++) x[u] = a[((size_t)(rg + RS * u) << 8) + col0 + c];
    } else {
        constexpr int V = 1 << R2;
#pragma unroll
        for (int k = 0; k < (256 >> C); k++) {
            const int item = tid + T * k;
            const int c2 = item & 15, grp = item >> 4;
            u64 y[V];
#pragma unroll
            for (int v = 0; v < V; v++) y[v] = a[((size_t)((grp << R2) + v) << 8) + col0 + c2];
#pragma unroll
            for (int st = 0; st < R2; st++) {
                const int b = st;
#pragma unroll
                for (int v = 0; v < V; v++) {
                    if (v >> st & 1) continue;
                    gs_bfly<LZ>(y[v], y[v | (1 << st)],
                                ldtw(tw, (1 << (LOGN - 9 - b)) + ((grp << R2) >> (b + 1)) + (v >> (b + 1))), mc.q,
                                mc.two_q, mc.two_q << (b + 8));
                }
            }
#pragma unroll
            for (int v = 0; v < V; v++) s[(((grp << R2) + v) << 4) + c2] = y[v];
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 16; u++) x[u] = s[((rg + RS * u) << 4) + c];
    }
#pragma unroll
    for (int st = 0; st < 4; st++) {
        const int b = R2 + st;
#pragma unroll
        for (int u = 0; u < 16; u++) {
            if (u >> st & 1) continue;
            if (st == 3) {
                // final stage (t = N/2): (x + y) N^-1 and (x - y) psi^{-br(1)} N^-1, fully reduced
                const u64 xa = x[u] + x[u | 8];
                const u64 xb = x[u] + (LZ ? (mc.two_q << (b + 8)) : mc.two_q) - x[u | 8];
                const ulonglong2 wl = ldtw(tw, 0);
                x[u] = mul_shoup(xa, mc.n_inv, mc.n_inv_sh, mc.q);
                x[u | 8] = mul_shoup(xb, wl.x, wl.y, mc.q);
            } else {
                gs_bfly<LZ>(x[u], x[u | (1 << st)], ldtw(tw, (1 << (LOGN - 9 - b)) + (u >> (b + 1 - R2))), mc.q,
                            mc.two_q, mc.two_q << (b + 8));
            }
        }
    }
#pragma unroll
    for (int u = 0; u < 16; u++) a[((size_t)(rg + RS * u) << 8) + col0 + c] = x[u];
}

template <int C, int MINB>
__global__ void __launch_bounds__(1 << C, MINB) ntt_inv_col(u64* base, size_t batch_stride, RowMap map, NttTables tb) {
    constexpr int LOGN = C + 8;
    __shared__ u64 s[C > 4 ? (16 << C) : 1];
    int mi;
    u64* a = limb_ptr(base, batch_stride, map, blockIdx.y, LOGN, mi);
    const ModConst mc = tb.mc[mi];
    const ulonglong2* tw = tb.inv + ((size_t)mi << LOGN);
    if (mc.q < kLazyLimit)
        inv_col_body<C, true>(a, s, mc, tw, blockIdx.x * 16);
    else
        inv_col_body<C, false>(a, s, mc, tw, blockIdx.x * 16);
}

// ------------------------------------------------------------------------------ row pass
// forward: bits 7 .. 0 inside 256-word blocks; output fully reduced to [0, q)
// in: the CTA's 8 blocks (global memory, or a shared-memory copy that `s` may alias: then
// SYNC_IN makes every thread finish reading before the first exchange); a: the output blocks
template <bool LZ, bool SYNC_IN = false>
__device__ __forceinline__ void fwd_row_body(const u64* in, u64* a, u64* s, const ModConst& mc, const ulonglong2* tw,
                                             int log_n, int g_blk) {
    const int tid = threadIdx.x;
    const int lo = tid & 15, blk = tid >> 4;
    const int g0 = g_blk + (blk << 8);
    u64 x[16];
#pragma unroll
    for (int u = 0; u < 16; u++) x[u] = in[(blk << 8) + lo + 16 * u];
    if (SYNC_IN) __syncthreads();
#pragma unroll
    for (int st = 3; st >= 0; st--) {
        const int b = 4 + st;
#pragma unroll
        for (int u = 0; u < 16; u++) {
            if (u >> st & 1) continue;
            // j = g0 + lo + 16u, g0 a multiple of 256, lo < 16: j >> (b+1) = (g0 >> (b+1)) + (u >> (b-3))
            ct_bfly<LZ>(x[u], x[u | (1 << st)], ldtw(tw, (1 << (log_n - 1 - b)) + (g0 >> (b + 1)) + (u >> (b - 3))),
                        mc.q, mc.two_q);
        }
    }
#pragma unroll
    for (int u = 0; u < 16; u++) s[swz((blk << 8) + lo + 16 * u)] = x[u];
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 16; u++) x[u] = s[swz((blk << 8) + 16 * lo + u)];
#pragma unroll
    for (int st = 3; st >= 0; st--) {
        const int b = st;
#pragma unroll
        for (int u = 0; u < 16; u++) {
            if (u >> st & 1) continue;
            // twiddle (g0 + 16 lo + u) >> (b+1) of the stage, stored lane-interleaved (tw_row_slot)
            ct_bfly<LZ>(x[u], x[u | (1 << st)], ldtw(tw, tw_row_slot(log_n, b, g0, lo, u)), mc.q, mc.two_q);
        }
    }
#pragma unroll
    for (int u = 0; u < 16; u++)
        s[swz((blk << 8) + 16 * lo + u)] = LZ ? reduce_lazy(x[u], mc) : csub(csub(x[u], mc.two_q), mc.q);
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 16; u++) a[(blk << 8) + lo + 16 * u] = s[swz((blk << 8) + lo + 16 * u)];
}

template <int LOGN, int MINB>
__global__ void __launch_bounds__(kRowThreads, MINB) ntt_fwd_row(u64* base, size_t batch_stride, RowMap map,
                                                              NttTables tb) {
    constexpr int log_n = LOGN;
    constexpr int E = 8 * 256;
    __shared__ u64 s[E];
    int mi;
    u64* a = limb_ptr(base, batch_stride, map, blockIdx.y, log_n, mi) + (size_t)blockIdx.x * E;
    const ModConst mc = tb.mc[mi];
    const ulonglong2* tw = tb.fwd + ((size_t)mi << log_n);
    if (mc.q < kLazyLimit)
        fwd_row_body<true>(a, a, s, mc, tw, log_n, blockIdx.x * E);
    else
        fwd_row_body<false>(a, a, s, mc, tw, log_n, blockIdx.x * E);
}

// Persistent form of the forward row pass: each block walks tiles (limb, 8 blocks of 256 words)
// with stride gridDim.x; one thread streams the NEXT tile into the other half of a double
// buffer with a bulk copy (TMA) while the block transforms the current one, so the global-load
// latency of a tile overlaps the previous tile's butterflies.  The current tile's buffer also
// serves as the exchange buffer.  A tile that does not arrive within the poll limit makes the
// whole block stop (block-wide vote) and report LC_ERR_TIMEOUT.
template <int MINB>
__global__ void __launch_bounds__(kRowThreads, MINB) ntt_fwd_row_tma(u64* base, size_t batch_stride, RowMap map,
                                                                  int log_n, NttTables tb, int total_tiles) {
    constexpr int E = 8 * 256;
    constexpr unsigned BYTES = E * 8;
    __shared__ __align__(128) u64 buf[2][E];
    __shared__ __align__(8) uint64_t bar[2];
    const int tiles_per_limb = (1 << log_n) / E;
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    int mi;
    int tile = blockIdx.x;
    if (tid == 0 && tile < total_tiles) {
        const int b = tile / tiles_per_limb;
        const u64* src = limb_ptr(base, batch_stride, map, b, log_n, mi) + (size_t)(tile - b * tiles_per_limb) * E;
        mbar_arrive_expect_tx(&bar[0], BYTES);
        bulk_load(buf[0], src, BYTES, &bar[0]);
    }
    for (int i = 0; tile < total_tiles; i++, tile += gridDim.x) {
        const int nxt = tile + gridDim.x;
        const bool more = nxt < total_tiles;
        if (tid == 0 && more) {  // the other buffer was released by the barrier ending iteration i-1
            fence_proxy_async();
            const int b = nxt / tiles_per_limb;
            const u64* src = limb_ptr(base, batch_stride, map, b, log_n, mi) + (size_t)(nxt - b * tiles_per_limb) * E;
            mbar_arrive_expect_tx(&bar[(i + 1) & 1], BYTES);
            bulk_load(buf[(i + 1) & 1], src, BYTES, &bar[(i + 1) & 1]);
        }
        const int b = tile / tiles_per_limb;
        u64* a = limb_ptr(base, batch_stride, map, b, log_n, mi) + (size_t)(tile - b * tiles_per_limb) * E;
        if (!__syncthreads_and(mbar_wait(&bar[i & 1], (i >> 1) & 1))) {
            if (tid == 0) {
                atomicOr(tb.err, LC_ERR_TIMEOUT);
                if (more) mbar_wait(&bar[(i + 1) & 1], ((i + 1) >> 1) & 1);  // let the copy in flight land
            }
            return;
        }
        const ModConst mc = tb.mc[mi];
        const ulonglong2* tw = tb.fwd + ((size_t)mi << log_n);
        const int g_blk = (tile - b * tiles_per_limb) * E;
        if (mc.q < kLazyLimit)
            fwd_row_body<true, true>(buf[i & 1], a, buf[i & 1], mc, tw, log_n, g_blk);
        else
            fwd_row_body<false, true>(buf[i & 1], a, buf[i & 1], mc, tw, log_n, g_blk);
        __syncthreads();  // this buffer is free for the copy issued two tiles later
    }
}

// inverse: bits 0 .. 7 inside 256-word blocks (global stages 0 .. 7), input in [0, 2q)
template <bool LZ>
__device__ __forceinline__ void inv_row_body(u64* a, u64* s, const ModConst& mc, const ulonglong2* tw, int log_n,
                                             int g_blk) {
    const int tid = threadIdx.x;
    const int lo = tid & 15, blk = tid >> 4;
    const int g0 = g_blk + (blk << 8);
    u64 x[16];
#pragma unroll
    for (int u = 0; u < 16; u++) s[swz((blk << 8) + lo + 16 * u)] = a[(blk << 8) + lo + 16 * u];
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 16; u++) x[u] = s[swz((blk << 8) + 16 * lo + u)];
#pragma unroll
    for (int st = 0; st < 4; st++) {
        const int b = st;
#pragma unroll
        for (int u = 0; u < 16; u++) {
            if (u >> st & 1) continue;
            gs_bfly<LZ>(x[u], x[u | (1 << st)], ldtw(tw, tw_row_slot(log_n, b, g0, lo, u)), mc.q, mc.two_q,
                        mc.two_q << b);
        }
    }
#pragma unroll
    for (int u = 0; u < 16; u++) s[swz((blk << 8) + 16 * lo + u)] = x[u];
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 16; u++) x[u] = s[swz((blk << 8) + lo + 16 * u)];
#pragma unroll
    for (int st = 0; st < 4; st++) {
        const int b = 4 + st;
#pragma unroll
        for (int u = 0; u < 16; u++) {
            if (u >> st & 1) continue;
            gs_bfly<LZ>(x[u], x[u | (1 << st)], ldtw(tw, (1 << (log_n - 1 - b)) + (g0 >> (b + 1)) + (u >> (b - 3))),
                        mc.q, mc.two_q, mc.two_q << b);
        }
    }
#pragma unroll
    for (int u = 0; u < 16; u++) a[(blk << 8) + lo + 16 * u] = x[u];
}

template <int LOGN, int MINB>
__global__ void __launch_bounds__(kRowThreads, MINB) ntt_inv_row(u64* base, size_t batch_stride, RowMap map,
                                                              NttTables tb) {
    constexpr int log_n = LOGN;
    constexpr int E = 8 * 256;
    __shared__ u64 s[E];
    int mi;
    u64* a = limb_ptr(base, batch_stride, map, blockIdx.y, log_n, mi) + (size_t)blockIdx.x * E;
    const ModConst mc = tb.mc[mi];
    const ulonglong2* tw = tb.inv + ((size_t)mi << log_n);
    if (mc.q < kLazyLimit)
        inv_row_body<true>(a, s, mc, tw, log_n, blockIdx.x * E);
    else
        inv_row_body<false>(a, s, mc, tw, log_n, blockIdx.x * E);
}

}  // namespace

// column pass: C = log_n - 8 in [4, 8]; MINB (minimum resident blocks, i.e. a register cap) is
// a tuning choice: 1, 6, 7 or 8
#define LC_COL_C(KERNEL, MB, C_, GRID, S_)                                                          \
    switch (C_) {                                                                                   \
        case 4: KERNEL<4, MB><<<GRID, 1 << 4, 0, S_>>>(base, batch_stride, map, tb); break;         \
        case 5: KERNEL<5, MB><<<GRID, 1 << 5, 0, S_>>>(base, batch_stride, map, tb); break;         \
        case 6: KERNEL<6, MB><<<GRID, 1 << 6, 0, S_>>>(base, batch_stride, map, tb); break;         \
        case 7: KERNEL<7, MB><<<GRID, 1 << 7, 0, S_>>>(base, batch_stride, map, tb); break;         \
        case 8: KERNEL<8, MB><<<GRID, 1 << 8, 0, S_>>>(base, batch_stride, map, tb); break;         \
        default: break;                                                                             \
    }
#define LC_COL_DISPATCH(KERNEL, MINB_, C_, GRID, S_)            \
    switch (MINB_) {                                            \
        case 6: LC_COL_C(KERNEL, 6, C_, GRID, S_) break;        \
        case 7: LC_COL_C(KERNEL, 7, C_, GRID, S_) break;        \
        case 8: LC_COL_C(KERNEL, 8, C_, GRID, S_) break;        \
        default: LC_COL_C(KERNEL, 1, C_, GRID, S_) break;       \
    }
// row pass: log_n in [12, 16] (a compile-time ring degree), MINB 4, 5 or 6
#define LC_ROW_N(KERNEL, MB, LOGN_, GRID, S_)                                                      \
    switch (LOGN_) {                                                                               \
        case 12: KERNEL<12, MB><<<GRID, kRowThreads, 0, S_>>>(base, batch_stride, map, tb); break; \
        case 13: KERNEL<13, MB><<<GRID, kRowThreads, 0, S_>>>(base, batch_stride, map, tb); break; \
        case 14: KERNEL<14, MB><<<GRID, kRowThreads, 0, S_>>>(base, batch_stride, map, tb); break; \
        case 15: KERNEL<15, MB><<<GRID, kRowThreads, 0, S_>>>(base, batch_stride, map, tb); break; \
        case 16: KERNEL<16, MB><<<GRID, kRowThreads, 0, S_>>>(base, batch_stride, map, tb); break; \
        default: break;                                                                            \
    }
#define LC_ROW_DISPATCH(KERNEL, MINB_, GRID, S_)                   \
    switch (MINB_) {                                               \
        case 4: LC_ROW_N(KERNEL, 4, log_n, GRID, S_) break;        \
        case 6: LC_ROW_N(KERNEL, 6, log_n, GRID, S_) break;        \
        default: LC_ROW_N(KERNEL, 5, log_n, GRID, S_) break;       \
    }

// Register-resident copy of the forward butterfly network: radix-16 blocks of the lazy
// Cooley-Tukey butterfly (the 40-bit-prime path of the transforms above) with twiddles held in
// registers, so that the butterfly arithmetic runs without memory traffic or exchanges.  The
// values wrap modulo 2^64 instead of staying reduced; the instruction stream is the same.
__global__ void __launch_bounds__(kProbeThreads) ntt_bfly_probe(u64 q, u64 w, u64 w_sh, uint32_t iters,
                                                                unsigned long long* sink) {
    u64 x[16];
#pragma unroll
    for (int u = 0; u < 16; u++) x[u] = (u64)threadIdx.x * 16 + u + blockIdx.x;
    ulonglong2 tw[4];
#pragma unroll
    for (int k = 0; k < 4; k++) tw[k] = make_ulonglong2(w + 2 * k, w_sh - 2 * k);
    for (uint32_t it = 0; it < iters; it++) {
#pragma unroll
        for (int st = 3; st >= 0; st--) {
#pragma unroll
            for (int u = 0; u < 16; u++) {
                if (u >> st & 1) continue;
                ct_bfly<true>(x[u], x[u | (1 << st)], tw[st], q, 2 * q);
            }
        }
    }
    u64 acc = 0;
#pragma unroll
    for (int u = 0; u < 16; u++) acc ^= x[u];
    if (acc == 0x9e3779b97f4a7c15ull) atomicAdd(sink, 1ull);
}

void probe_ntt_bfly(int blocks, uint32_t iters, unsigned long long* sink, cudaStream_t s) {
    // the largest 40-bit prime q = 1 mod 2^16, and a Shoup pair for one of its residues
    const u64 q = 1099510054913ull, w = 0x5f3759df12ull % q;
    const u64 w_sh = (u64)(((unsigned __int128)w << 64) / q);
    ntt_bfly_probe<<<blocks, kProbeThreads, 0, s>>>(q, w, w_sh, iters, sink);
}

// persistent grid of a row-pass kernel: resident blocks per SM x SMs (queried once per kernel
// and device)
template <typename K>
static int persistent_grid(K kernel, int total) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    const auto key = std::make_pair(reinterpret_cast<const void*>(kernel), dev);
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    int cap;
    if (it != cache.end()) {
        cap = it->second;
    } else {
        int sms = 0, per = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, kRowThreads, 0);
        cap = std::max(1, sms * std::max(1, per));
        cache[key] = cap;
    }
    return std::min(total, cap);
}

void ntt_forward(u64* base, size_t batch_stride, int batch, const RowMap& map, int log_n, const NttTables& tb,
                 cudaStream_t s, NttTune tune) {
    const int limbs = batch * map.n;
    if (limbs == 0) return;
    const int C = log_n - 8;
    dim3 gc(16, limbs), gr((1 << log_n) / 2048, limbs);
    LC_COL_DISPATCH(ntt_fwd_col, tune.col_minb, C, gc, s)
    if (tune.row_tma) {
        const int total = limbs * ((1 << log_n) / 2048);
        switch (tune.row_minb) {
            case 4: {
                const int g = persistent_grid(ntt_fwd_row_tma<4>, total);
                ntt_fwd_row_tma<4><<<g, kRowThreads, 0, s>>>(base, batch_stride, map, log_n, tb, total);
                break;
            }
            case 6: {
                const int g = persistent_grid(ntt_fwd_row_tma<6>, total);
                ntt_fwd_row_tma<6><<<g, kRowThreads, 0, s>>>(base, batch_stride, map, log_n, tb, total);
                break;
            }
            default: {
                const int g = persistent_grid(ntt_fwd_row_tma<5>, total);
                ntt_fwd_row_tma<5><<<g, kRowThreads, 0, s>>>(base, batch_stride, map, log_n, tb, total);
                break;
            }
        }
    } else {
        LC_ROW_DISPATCH(ntt_fwd_row, tune.row_minb, gr, s)
    }
    g_lc_launches += 2;
}

void ntt_inverse(u64* base, size_t batch_stride, int batch, const RowMap& map, int log_n, const NttTables& tb,
                 cudaStream_t s, NttTune tune) {
    const int limbs = batch * map.n;
    if (limbs == 0) return;
    const int C = log_n - 8;
    dim3 gc(16, limbs), gr((1 << log_n) / 2048, limbs);
    LC_ROW_DISPATCH(ntt_inv_row, tune.row_minb, gr, s)
    LC_COL_DISPATCH(ntt_inv_col, tune.col_minb, C, gc, s)
    g_lc_launches += 2;
}

// Device modular arithmetic for word-size RNS primes q < 2^62.
//
// Shoup multiplication (V. Shoup, NTL; D. Harvey, "Faster arithmetic for number-theoretic
// transforms", 2014): with w' = floor(w 2^64 / q), for any a < 2^64
//   a*w - floor(a w' / 2^64) * q  lies in [0, 2q).
// 128-bit values are reduced as hi*(2^64 mod q) + lo, each term by a Shoup product.
#pragma once
#include <cstdint>

typedef uint64_t u64;

struct ModConst {
    u64 q;        // the prime
    u64 two_q;
    u64 r64;      // 2^64 mod q
    u64 r64_sh;   // floor(r64 * 2^64 / q)
    u64 one_sh;   // floor(2^64 / q)
    u64 n_inv;    // N^-1 mod q
    u64 n_inv_sh;
    // final reduction of lazy transform values (reduce_lazy below): bits 0..31 c = floor(2^(b+31)/q)
    // with b = bits(q); bits 32..39 s1 = max(0, b - 26); bits 40..47 sh = b + 31 - s1
    u64 lzr;
};

// x mod q for x < 64 q (the lazy range of the transforms for primes below 2^46), in [0, q).
// xh = floor(x / 2^s1) < 2^32 and t = floor(xh c / 2^sh) approximate x / q from below: the
// truncation of x loses < 2^s1 / q <= 2^-25 and that of c < xh 2^s1 / 2^(b+31) < 2^-25 of a
// quotient unit, so t is floor(x / q) or one less, x - t q lies in [0, 2q) and one
// conditional subtraction finishes.
__device__ __forceinline__ u64 reduce_lazy(u64 x, const ModConst& m) {
    const unsigned c = (unsigned)m.lzr, s1 = (unsigned)(m.lzr >> 32) & 255u, sh = (unsigned)(m.lzr >> 40) & 255u;
    const unsigned xh = (unsigned)(x >> s1);
    const unsigned t = (unsigned)(((u64)xh * c) >> sh);
    const u64 r = x - (u64)t * m.q;
    return r >= m.q ? r - m.q : r;
}

__device__ __forceinline__ u64 mul_shoup_lazy(u64 a, u64 w, u64 w_sh, u64 q) {
    u64 hi = __umul64hi(a, w_sh);
    return a * w - hi * q;  // [0, 2q)
}

__device__ __forceinline__ u64 csub(u64 a, u64 m) { return a >= m ? a - m : a; }

__device__ __forceinline__ u64 mul_shoup(u64 a, u64 w, u64 w_sh, u64 q) {
    return csub(mul_shoup_lazy(a, w, w_sh, q), q);
}

__device__ __forceinline__ u64 add_mod(u64 a, u64 b, u64 q) { return csub(a + b, q); }
__device__ __forceinline__ u64 sub_mod(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + q - b; }

// 128-bit accumulator helpers
struct u128v {
    u64 lo, hi;
};
// acc += a * b (128-bit), one carry chain
__device__ __forceinline__ void mac128(u128v& acc, u64 a, u64 b) {
    asm("mad.lo.cc.u64 %0, %2, %3, %0;\n\t"
        "madc.hi.u64 %1, %2, %3, %1;"
        : "+l"(acc.lo), "+l"(acc.hi)
        : "l"(a), "l"(b));
}
// acc += v (64-bit addend)
__device__ __forceinline__ void add128(u128v& acc, u64 v) {
    asm("add.cc.u64 %0, %0, %2;\n\t"
        "addc.u64 %1, %1, 0;"
        : "+l"(acc.lo), "+l"(acc.hi)
        : "l"(v));
}
// (hi * 2^64 + lo) mod q in [0, q) for any hi, lo
__device__ __forceinline__ u64 reduce128(u128v x, const ModConst& m) {
    u64 a = mul_shoup_lazy(x.hi, m.r64, m.r64_sh, m.q);  // [0, 2q)
    u64 b = x.lo - __umul64hi(x.lo, m.one_sh) * m.q;     // [0, 2q)
    u64 s = a + b;                                       // [0, 4q)
    s = csub(s, m.two_q);
    return csub(s, m.q);
}
__device__ __forceinline__ u64 mul_mod(u64 a, u64 b, const ModConst& m) {
    u128v t{a * b, __umul64hi(a, b)};
    return reduce128(t, m);
}
// centred lift of a residue of an odd modulus p into another modulus q (as a residue)
__device__ __forceinline__ u64 lift_centred(u64 v, u64 p, u64 q) {
    // v in [0, p): if v > (p-1)/2 the integer is v - p < 0
    if (v > (p >> 1)) {
        u64 neg = p - v;  // in [1, p/2]
        neg = neg % q;    // p may exceed q
        return neg ? q - neg : 0;
    }
    return v % q;
}

// (hi * 2^64 + lo) mod q in [0, q), constants given explicitly (q < 2^62)
__device__ __forceinline__ u64 reduce128c(u128v x, u64 q, u64 r64, u64 r64_sh, u64 one_sh) {
    u64 a = mul_shoup_lazy(x.hi, r64, r64_sh, q);
    u64 b = x.lo - __umul64hi(x.lo, one_sh) * q;
    u64 s = a + b;
    s = csub(s, 2 * q);
    return csub(s, q);
}

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
    // with b = bits(q); bits 32..39 s1 = max(0, b - 25); bits 40..47 sh = b + 31 - s1
    u64 lzr;
};

// x mod q for x < 128 q (the lazy range of the transforms for primes below 2^46), in [0, q).
// xh = floor(x / 2^s1) < 2^32 and t = floor(xh c / 2^sh) approximate x / q from below: the
// truncation of x loses < 2^s1 / q <= 2^-24 and that of c < xh 2^s1 / 2^(b+31) < 2^-24 of a
// quotient unit, so t is floor(x / q) or one less, x - t q lies in [0, 2q) and one
// conditional subtraction finishes.
__device__ __forceinline__ u64 reduce_lazy(u64 x, const ModConst& m) {
    const unsigned c = (unsigned)m.lzr, s1 = (unsigned)(m.lzr >> 32) & 255u, sh = (unsigned)(m.lzr >> 40) & 255u;
    const unsigned xh = (unsigned)(x >> s1);
    const unsigned t = (unsigned)(((u64)xh * c) >> sh);
    const u64 r = x - (u64)t * m.q;
    return r >= m.q ? r - m.q : r;
}

// y w + t n mod 2^64 as one chain of 32-bit multiply-adds (with n = 2^64 - q: y w - t q, the
// remainder step of a Shoup product).  Written out because the chain of eight 32-bit products
// with one carry measured faster than two 64-bit products and a 64-bit subtraction (8-9 % more
// butterflies per second in a register-resident transform butterfly).
__device__ __forceinline__ u64 mul_sub_lo(u64 y, u64 w, u64 t, u64 n) {
    unsigned r0, r1;
    asm("{\n\t"
        ".reg .u32 y0, y1, w0, w1, t0, t1, n0, n1;\n\t"
        "mov.b64 {y0, y1}, %2;\n\t"
        "mov.b64 {w0, w1}, %3;\n\t"
        "mov.b64 {t0, t1}, %4;\n\t"
        "mov.b64 {n0, n1}, %5;\n\t"
        "mul.lo.u32 %0, y0, w0;\n\t"
        "mul.hi.u32 %1, y0, w0;\n\t"
        "mad.lo.u32 %1, y1, w0, %1;\n\t"
        "mad.lo.u32 %1, y0, w1, %1;\n\t"
        "mad.lo.cc.u32 %0, t0, n0, %0;\n\t"
        "madc.hi.u32 %1, t0, n0, %1;\n\t"
        "mad.lo.u32 %1, t1, n0, %1;\n\t"
        "mad.lo.u32 %1, t0, n1, %1;\n\t"
        "}"
        : "=&r"(r0), "=&r"(r1)
        : "l"(y), "l"(w), "l"(t), "l"(n));
    return ((u64)r1 << 32) | r0;
}

__device__ __forceinline__ u64 mul_shoup_lazy(u64 a, u64 w, u64 w_sh, u64 q) {
    return mul_sub_lo(a, w, __umul64hi(a, w_sh), 0 - q);  // a w - floor(a w' / 2^64) q, in [0, 2q)
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
// acc += a * b (mod 2^128).  Written with the compiler's 128-bit integers: measured 1.24x the
// multiply-adds per second of a 64-bit mad.lo.cc / madc.hi pair in a register-resident loop.
__device__ __forceinline__ void mac128(u128v& acc, u64 a, u64 b) {
    const unsigned __int128 s = ((unsigned __int128)acc.hi << 64 | acc.lo) + (unsigned __int128)a * b;
    acc.lo = (u64)s;
    acc.hi = (u64)(s >> 64);
}
// acc += v (64-bit addend)
__device__ __forceinline__ void add128(u128v& acc, u64 v) {
    const unsigned __int128 s = ((unsigned __int128)acc.hi << 64 | acc.lo) + v;
    acc.lo = (u64)s;
    acc.hi = (u64)(s >> 64);
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

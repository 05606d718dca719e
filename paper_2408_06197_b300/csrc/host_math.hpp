// Host-side number theory for building the library's device tables.
#pragma once
#include <cstdint>
#include <vector>

namespace lc {

typedef uint64_t u64;
typedef unsigned __int128 u128;

inline u64 hmul(u64 a, u64 b, u64 m) { return (u64)((u128)a * b % m); }

inline u64 hpow(u64 base, u64 e, u64 m) {
    u64 acc = 1 % m;
    base %= m;
    for (; e; e >>= 1) {
        if (e & 1) acc = hmul(acc, base, m);
        base = hmul(base, base, m);
    }
    return acc;
}

inline u64 hinv(u64 a, u64 m) { return hpow(a % m, m - 2, m); }  // m prime

// floor(w * 2^64 / q) for w < q
inline u64 shoup_of(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }

// Miller-Rabin, deterministic for 64-bit inputs with the first twelve prime bases.
inline bool probable_prime(u64 n) {
    if (n < 4) return n == 2 || n == 3;
    const u64 bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    for (u64 b : bases)
        if (n % b == 0) return n == b;
    int r = 0;
    u64 d = n - 1;
    while (!(d & 1)) {
        d >>= 1;
        ++r;
    }
    for (u64 b : bases) {
        u64 x = hpow(b, d, n);
        if (x == 1 || x == n - 1) continue;
        int i = 1;
        for (; i < r; ++i) {
            x = hmul(x, x, n);
            if (x == n - 1) break;
        }
        if (i == r) return false;
    }
    return true;
}

// The `count` largest primes below 2^bits (and at least 2^(bits-1)) congruent to 1 mod 2N,
// after skipping the first `skip`, in descending order.
inline bool ntt_primes(int log_n, int bits, int skip, int count, std::vector<u64>& out) {
    const u64 step = (u64)2 << log_n;
    const u64 hi = (bits >= 64) ? ~(u64)0 : ((u64)1 << bits) - 1;
    const u64 lo = (u64)1 << (bits - 1);
    u64 v = hi - (hi - 1) % step;  // largest value <= hi with v = 1 mod step
    out.clear();
    int seen = 0;
    while ((int)out.size() < count) {
        if (v < lo || v <= step) return false;
        if (probable_prime(v)) {
            if (seen >= skip) out.push_back(v);
            ++seen;
        }
        v -= step;
    }
    return true;
}

// a primitive 2N-th root of unity mod q (q = 1 mod 2N): x^((q-1)/2N) for the first x >= 3
// whose power has order exactly 2N (checked as w^N = -1)
inline u64 root_2n(u64 q, int log_n) {
    const u64 n = (u64)1 << log_n;
    for (u64 x = 3;; ++x) {
        u64 w = hpow(x, (q - 1) / (2 * n), q);
        if (hpow(w, n, q) == q - 1) return w;
    }
}

inline unsigned bit_reverse(unsigned x, int bits) {
    unsigned r = 0;
    for (int i = 0; i < bits; ++i) r |= ((x >> i) & 1u) << (bits - 1 - i);
    return r;
}

}  // namespace lc

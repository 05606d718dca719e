"""The value-range arguments the transform kernels rely on, checked in exact integer arithmetic
on the host (no GPU): the three-partial-product Shoup quotient used for primes below 2^46, the
lazy ranges of both butterflies, and the final reduction's quotient estimate.  These restate the
arguments of the kernels' comments as checks; the kernels themselves are compared with the
oracle bit for bit in the GPU tests."""
import random

M32, M64 = (1 << 32) - 1, (1 << 64) - 1


def _is_prime(n):
    if n < 2:
        return False
    for p in (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37):
        if n % p == 0:
            return n == p
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37):
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def _primes():
    """The largest 30-, 40- and 45-bit primes = 1 mod 2^17 (NTT-friendly up to N = 2^16, all below
    the 2^46 limit of the lazy discipline)."""
    out = []
    for bits in (30, 40, 45):
        q = (1 << bits) - (1 << 17) + 1
        while not _is_prime(q):
            q -= 1 << 17
        out.append(q)
    return out


def quotient3(y, w_sh):
    """floor(y w' / 2^64) from the partial products y1 w'1, hi32(y0 w'1), hi32(y1 w'0)."""
    y0, y1 = y & M32, y >> 32
    p0, p1 = w_sh & M32, w_sh >> 32
    return y1 * p1 + ((y0 * p1) >> 32) + ((y1 * p0) >> 32)


def _samples(q, rng, n=4000):
    for k in range(n):
        w = q - 1 if k % 7 == 0 else rng.randrange(q)
        if k % 3 == 0:
            y = M64 - rng.randrange(1 << 16)  # the top of the 64-bit range
        elif k % 3 == 1:
            y = 68 * q - 1 - rng.randrange(1 << 10)  # the top of the forward lazy range
        else:
            y = rng.randrange(1 << 64)
        yield y, w


def test_three_product_quotient_is_at_most_two_short():
    rng = random.Random(5)
    for q in _primes():
        assert q < 1 << 46
        for y, w in _samples(q, rng):
            w_sh = (w << 64) // q
            t = quotient3(y, w_sh)
            exact = (y * w_sh) >> 64
            assert exact - 2 <= t <= exact
            r = (y * w - t * q) & M64  # what the kernel computes modulo 2^64
            assert r == y * w - t * q  # no wrap: the true value is non-negative and small
            assert 0 <= r < 4 * q and r % q == y * w % q


def test_forward_lazy_range_stays_below_128q():
    """Cooley-Tukey with products in [0, 4q) and no reduction: inputs below 4q grow by less than
    4q per stage; after log2(N) <= 16 stages they stay below 68q (inside the final reduction's
    128q), and below 2^64."""
    for q in _primes():
        bound = 4 * q
        for _ in range(16):
            bound = bound + 4 * q  # x + t and x + 4q - t, t in [0, 4q)
        assert bound <= 68 * q < 128 * q < 1 << 64


def test_inverse_lazy_range_fits_the_subtracted_multiples():
    """Gentleman-Sande with products in [0, 4q): inputs below 2q; at stage b every value is below
    2^(b+1) q, the multiple the kernels add before subtracting, and both outputs of the stage's
    additions stay below 2^(b+2) q < 2^64 up to log2(N) = 16."""
    for q in _primes():
        for log_n in (15, 16):
            bound = 2 * q  # inputs
            for b in range(log_n):
                ky = (2 * q) << b
                assert bound <= ky  # x + ky - y does not wrap
                assert bound + ky <= 2 * ky < 1 << 64  # x + y and x + ky - y
                bound = max(2 * bound, 4 * q)  # sums double; products are below 4q


def test_final_reduction_estimate_is_floor_or_one_less():
    """reduce_lazy: xh = floor(x / 2^s1), c = floor(2^(b+31) / q), t = floor(xh c / 2^sh) with
    s1 = max(0, b - 25), sh = b + 31 - s1 is floor(x / q) or one less for x < 128 q."""
    rng = random.Random(9)
    for q in _primes():
        b = q.bit_length()
        s1, sh = max(0, b - 25), b + 31 - max(0, b - 25)
        c = (1 << (b + 31)) // q
        assert c < 1 << 32
        for k in range(4000):
            x = 128 * q - 1 - rng.randrange(1 << 12) if k % 2 else rng.randrange(128 * q)
            xh = x >> s1
            assert xh < 1 << 32
            t = (xh * c) >> sh
            assert x // q - 1 <= t <= x // q
            r = x - t * q
            assert 0 <= r < 2 * q

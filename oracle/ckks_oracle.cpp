// TEST INFRASTRUCTURE ONLY -- plain CPU RNS-CKKS oracle for the Lancelot server evaluation.
//
// Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference legs may
// load this library.  It shares no code, header, table or constant generator with the
// CUDA library: every table here (primes, roots of unity, CRT constants) is recomputed
// from its definition with `unsigned __int128` and `%`.
//
// Representation (paper, "CKKS Scheme Description": RNS + double-CRT): a polynomial at
// level l is stored as (l+1) residue rows of N words; ciphertext polynomials live in the
// evaluation ("NTT") domain of THIS file's transform: row[k] = a(psi^(2k+1)) mod q, natural
// order, psi the first primitive 2N-th root found from 2 upward.  Interchange with the
// outside world is the coefficient domain (or_to_coeff / or_to_eval), which is independent
// of psi and ordering.
//
// Every step is exact integer arithmetic mod q except the points the method fixes:
// fast base conversion (ModUp/ModDown with centred representatives, no exact-CRT
// correction), rescale rounding (centred), and the order ModUp -> automorphism for rotations
// (hoisting, Section "Dynamic Hoisting").
//
// Parity status: pinned by tests/test_oracle_pins.py (big-integer checks on tiny N, NTT by
// direct evaluation, schoolbook convolution, exact rescale, ModUp/ModDown error sets,
// key-switch phase bound, decryption of products and rotations against plaintext).
#include <cstdint>
#include <cstring>
#include <cstdlib>
#include <vector>
#include <omp.h>

typedef uint64_t u64;
typedef int64_t i64;
typedef unsigned __int128 u128;

// ------------------------------------------------------------------ modular arithmetic
static inline u64 mul_mod(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }
static inline u64 add_mod(u64 a, u64 b, u64 q) { return (u64)(((u128)a + b) % q); }
static inline u64 sub_mod(u64 a, u64 b, u64 q) { return (u64)(((u128)(a % q) + q - (b % q)) % q); }
static u64 pow_mod(u64 b, u64 e, u64 q) {
    u64 r = 1 % q;
    b %= q;
    while (e) {
        if (e & 1) r = mul_mod(r, b, q);
        b = mul_mod(b, b, q);
        e >>= 1;
    }
    return r;
}
static u64 inv_mod(u64 a, u64 q) { return pow_mod(a % q, q - 2, q); }  // q prime
static inline u64 from_signed(i64 x, u64 q) {
    i64 r = x % (i64)q;
    if (r < 0) r += (i64)q;
    return (u64)r;
}

// deterministic Miller-Rabin for 64-bit integers (bases = first 12 primes)
static bool is_prime(u64 n) {
    if (n < 2) return false;
    static const u64 small[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    for (u64 p : small) {
        if (n % p == 0) return n == p;
    }
    u64 d = n - 1;
    int s = 0;
    while ((d & 1) == 0) { d >>= 1; s++; }
    for (u64 a : small) {
        u64 x = pow_mod(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int r = 1; r < s; r++) {
            x = mul_mod(x, x, n);
            if (x == n - 1) { comp = false; break; }
        }
        if (comp) return false;
    }
    return true;
}

// ------------------------------------------------------------------ context
struct OrCtx {
    int logN;
    size_t N;
    int nq, np, dnum, alpha;
    std::vector<u64> mod;                     // q_0..q_{nq-1}, p_0..p_{np-1}
    std::vector<u64> psi, n_inv;
    std::vector<std::vector<u64>> psi_pow, psi_inv_pow, om_pow, om_inv_pow;
    std::vector<size_t> bitrev;
    long long n_keyswitch = 0, n_modup = 0;
};

static int n_digits(const OrCtx& c, int level) { return (level + 1 + c.alpha - 1) / c.alpha; }

// textbook negacyclic NTT: weight by psi^i, bit-reverse, iterative radix-2 DFT with omega=psi^2.
// Output natural order: A[k] = sum_i a_i psi^{(2k+1) i} = a(psi^(2k+1)).
static void ntt_fwd(const OrCtx& c, int mi, u64* a) {
    const u64 q = c.mod[mi];
    const size_t N = c.N;
    for (size_t i = 0; i < N; i++) a[i] = mul_mod(a[i], c.psi_pow[mi][i], q);
    for (size_t i = 0; i < N; i++) {
        size_t j = c.bitrev[i];
        if (i < j) { u64 t = a[i]; a[i] = a[j]; a[j] = t; }
    }
    for (size_t len = 2; len <= N; len <<= 1) {
        size_t half = len / 2, step = N / len;
        for (size_t i = 0; i < N; i += len) {
            for (size_t j = 0; j < half; j++) {
                u64 u = a[i + j];
                u64 v = mul_mod(a[i + j + half], c.om_pow[mi][j * step], q);
                a[i + j] = add_mod(u, v, q);
                a[i + j + half] = sub_mod(u, v, q);
            }
        }
    }
}

static void ntt_inv(const OrCtx& c, int mi, u64* a) {
    const u64 q = c.mod[mi];
    const size_t N = c.N;
    for (size_t i = 0; i < N; i++) {
        size_t j = c.bitrev[i];
        if (i < j) { u64 t = a[i]; a[i] = a[j]; a[j] = t; }
    }
    for (size_t len = 2; len <= N; len <<= 1) {
        size_t half = len / 2, step = N / len;
        for (size_t i = 0; i < N; i += len) {
            for (size_t j = 0; j < half; j++) {
                u64 u = a[i + j];
                u64 v = mul_mod(a[i + j + half], c.om_inv_pow[mi][j * step], q);
                a[i + j] = add_mod(u, v, q);
                a[i + j + half] = sub_mod(u, v, q);
            }
        }
    }
    for (size_t i = 0; i < N; i++) a[i] = mul_mod(mul_mod(a[i], c.n_inv[mi], q), c.psi_inv_pow[mi][i], q);
}

// modulus index of row t of a polynomial over Q_level U P (rows 0..level are q, then p)
static inline int qp_mod_index(const OrCtx& c, int level, int t) { return t <= level ? t : c.nq + (t - level - 1); }

// automorphism X -> X^g on one coefficient-domain row (g odd): coefficient i moves to
// i*g mod 2N, negated when it lands in [N, 2N) because X^N = -1.
static void automorph_row(const OrCtx& c, const u64* in, u64* out, u64 q, u64 g) {
    const size_t N = c.N, twoN = 2 * N;
    for (size_t i = 0; i < N; i++) {
        size_t k = (size_t)(((u128)i * g) % twoN);
        if (k < N) out[k] = in[i] % q;
        else out[k - N] = (q - in[i] % q) % q;
    }
}

// ------------------------------------------------------------------ base conversion
// ModUp of digit j at level l (Section "Dynamic Hoisting", key-switching steps): for every
// row t of Q_l U P outside D_j: ext_t = sum_{i in D_j} y_i (D_j/q_i mod m_t) mod m_t with
// y_i = [c_i (D_j/q_i)^-1]_{q_i} taken as the CENTRED representative in (-q_i/2, q_i/2];
// rows inside D_j keep c_i.  Input and output are coefficient domain.  (The [0,q) representative
// would add a digit-mean bias that the key error concentrates at one slot.)
static void modup_digit(const OrCtx& c, const u64* c_coef, int level, int j, u64* ext) {
    const size_t N = c.N;
    const int nl = level + 1, rows = nl + c.np;
    const int lo = j * c.alpha, hi = std::min((j + 1) * c.alpha, nl);
    std::vector<u64> hat_inv(hi - lo);
    for (int i = lo; i < hi; i++) {
        u64 qi = c.mod[i], prod = 1 % qi;
        for (int k = lo; k < hi; k++)
            if (k != i) prod = mul_mod(prod, c.mod[k] % qi, qi);
        hat_inv[i - lo] = inv_mod(prod, qi);
    }
#pragma omp parallel for schedule(static) if (!omp_in_parallel())
    for (int t = 0; t < rows; t++) {
        u64* dst = ext + (size_t)t * N;
        if (t >= lo && t < hi) {
            std::memcpy(dst, c_coef + (size_t)t * N, N * sizeof(u64));
            continue;
        }
        const u64 mt = c.mod[qp_mod_index(c, level, t)];
        std::vector<u64> hat_t(hi - lo);
        for (int i = lo; i < hi; i++) {
            u64 prod = 1 % mt;
            for (int k = lo; k < hi; k++)
                if (k != i) prod = mul_mod(prod, c.mod[k] % mt, mt);
            hat_t[i - lo] = prod;
        }
        for (size_t x = 0; x < N; x++) {
            u64 acc = 0;
            for (int i = lo; i < hi; i++) {
                const u64 qi = c.mod[i];
                u64 y = mul_mod(c_coef[(size_t)i * N + x], hat_inv[i - lo], qi);
                i64 yc = y <= (qi - 1) / 2 ? (i64)y : (i64)y - (i64)qi;  // centred representative
                acc = add_mod(acc, mul_mod(from_signed(yc, mt), hat_t[i - lo], mt), mt);
            }
            dst[x] = acc;
        }
    }
}

// ModDown of one polynomial over Q_l U P given in the evaluation domain; output evaluation
// domain over Q_l: out_i = (u_i - sum_k y_k (P/p_k mod q_i)) * P^-1 mod q_i with
// y_k = [u_pk (P/p_k)^-1]_{p_k} taken as the centred representative.
static void moddown_eval(const OrCtx& c, const u64* u, int level, u64* out) {
    const size_t N = c.N;
    const int nl = level + 1, K = c.np;
    std::vector<u64> y((size_t)K * N);
    for (int k = 0; k < K; k++) {
        const int mk = c.nq + k;
        const u64 pk = c.mod[mk];
        u64 prod = 1 % pk;
        for (int m = 0; m < K; m++)
            if (m != k) prod = mul_mod(prod, c.mod[c.nq + m] % pk, pk);
        const u64 phat_inv = inv_mod(prod, pk);
        u64* yk = y.data() + (size_t)k * N;
        std::memcpy(yk, u + (size_t)(nl + k) * N, N * sizeof(u64));
        ntt_inv(c, mk, yk);
        for (size_t x = 0; x < N; x++) yk[x] = mul_mod(yk[x], phat_inv, pk);
    }
    // centred representatives y_k in (-p_k/2, p_k/2]; the conversion then approximates the
    // centred residue of u mod P, so ModDown rounds instead of flooring.
    auto centred = [&](int k, size_t x) -> i64 {
        const u64 pk = c.mod[c.nq + k], v = y[(size_t)k * N + x];
        return v <= (pk - 1) / 2 ? (i64)v : (i64)v - (i64)pk;
    };
#pragma omp parallel for schedule(static) if (!omp_in_parallel())
    for (int i = 0; i < nl; i++) {
        const u64 qi = c.mod[i];
        std::vector<u64> phat(K);
        u64 P_mod = 1 % qi;
        for (int k = 0; k < K; k++) {
            u64 prod = 1 % qi;
            for (int m = 0; m < K; m++)
                if (m != k) prod = mul_mod(prod, c.mod[c.nq + m] % qi, qi);
            phat[k] = prod;
            P_mod = mul_mod(P_mod, c.mod[c.nq + k] % qi, qi);
        }
        const u64 P_inv = inv_mod(P_mod, qi);
        std::vector<u64> conv(N);
        for (size_t x = 0; x < N; x++) {
            u64 acc = 0;
            for (int k = 0; k < K; k++) acc = add_mod(acc, mul_mod(from_signed(centred(k, x), qi), phat[k], qi), qi);
            conv[x] = acc;
        }
        ntt_fwd(c, i, conv.data());
        for (size_t x = 0; x < N; x++)
            out[(size_t)i * N + x] = mul_mod(sub_mod(u[(size_t)i * N + x], conv[x], qi), P_inv, qi);
    }
}

// coefficient-domain ModDown (pinning helper): input and output coefficient domain.
static void moddown_coef(const OrCtx& c, const u64* u_coef, int level, u64* out_coef) {
    const size_t N = c.N;
    const int nl = level + 1, rows = nl + c.np;
    std::vector<u64> u((size_t)rows * N);
    std::memcpy(u.data(), u_coef, u.size() * sizeof(u64));
    for (int t = 0; t < rows; t++) ntt_fwd(c, qp_mod_index(c, level, t), u.data() + (size_t)t * N);
    moddown_eval(c, u.data(), level, out_coef);
    for (int i = 0; i < nl; i++) ntt_inv(c, i, out_coef + (size_t)i * N);
}

// ------------------------------------------------------------------ key switching
// Hybrid key switching (Section "Dynamic Hoisting": decompose, ModUp, inner product with the
// key, ModDown).  For rotations the automorphism phi_g is applied to the extended digits
// AFTER ModUp (hoisted order); g = 1 means no automorphism (relinearisation).
// c_coef: coefficient domain [l+1][N]; keys[r]: evaluation domain [dnum][2][nq+np][N];
// out[r]: evaluation domain [2][l+1][N] (the switched pair before adding phi_g(c0)).
static void keyswitch_hoisted(OrCtx& c, const u64* c_coef, int level, int n_rot, const u64* gs,
                              const u64* const* keys, u64* const* outs, bool qp_sum = false) {
    const size_t N = c.N;
    const int nl = level + 1, rows = nl + c.np, beta = n_digits(c, level);
    std::vector<u64> ext((size_t)beta * rows * N);
    for (int j = 0; j < beta; j++) modup_digit(c, c_coef, level, j, ext.data() + (size_t)j * rows * N);
#pragma omp atomic
    c.n_modup += 1;
    // qp_sum: the inner products of all rotations are summed over Q_l U P and switched down
    // once (written to outs[0]); otherwise each rotation gets its own ModDown.
    std::vector<u64> u0((size_t)rows * N, 0), u1((size_t)rows * N, 0);
    for (int r = 0; r < n_rot; r++) {
        const u64 g = gs[r];
        if (!qp_sum) {
            std::fill(u0.begin(), u0.end(), 0);
            std::fill(u1.begin(), u1.end(), 0);
        }
#pragma omp parallel for schedule(static) if (!omp_in_parallel())
        for (int t = 0; t < rows; t++) {
            const int mi = qp_mod_index(c, level, t);
            const u64 m = c.mod[mi];
            const int kt = mi;  // key rows: q_0..q_{nq-1} then p_0..p_{np-1}
            std::vector<u64> e(N);
            for (int j = 0; j < beta; j++) {
                const u64* src = ext.data() + ((size_t)j * rows + t) * N;
                if (g == 1) std::memcpy(e.data(), src, N * sizeof(u64));
                else automorph_row(c, src, e.data(), m, g);
                ntt_fwd(c, mi, e.data());
                const u64* kb = keys[r] + (((size_t)j * 2 + 0) * (c.nq + c.np) + kt) * N;
                const u64* ka = keys[r] + (((size_t)j * 2 + 1) * (c.nq + c.np) + kt) * N;
                for (size_t x = 0; x < N; x++) {
                    u0[(size_t)t * N + x] = add_mod(u0[(size_t)t * N + x], mul_mod(e[x], kb[x], m), m);
                    u1[(size_t)t * N + x] = add_mod(u1[(size_t)t * N + x], mul_mod(e[x], ka[x], m), m);
                }
            }
        }
#pragma omp atomic
        c.n_keyswitch += 1;
        if (!qp_sum) {
            moddown_eval(c, u0.data(), level, outs[r]);
            moddown_eval(c, u1.data(), level, outs[r] + (size_t)nl * N);
        }
    }
    if (qp_sum) {
        moddown_eval(c, u0.data(), level, outs[0]);
        moddown_eval(c, u1.data(), level, outs[0] + (size_t)nl * N);
    }
}

static void to_coef(const OrCtx& c, u64* rows_data, int nrows) {
#pragma omp parallel for schedule(static) if (!omp_in_parallel())
    for (int i = 0; i < nrows; i++) ntt_inv(c, i, rows_data + (size_t)i * c.N);
}
static void to_eval(const OrCtx& c, u64* rows_data, int nrows) {
#pragma omp parallel for schedule(static) if (!omp_in_parallel())
    for (int i = 0; i < nrows; i++) ntt_fwd(c, i, rows_data + (size_t)i * c.N);
}

// relinearisation (Section "Lazy Relinearization"): (d0, d1) + KS(d2, rlk)
static void relin(OrCtx& c, const u64* ct3, int level, const u64* rlk, u64* out) {
    const size_t N = c.N;
    const int nl = level + 1;
    const size_t P = (size_t)nl * N;
    std::vector<u64> d2(ct3 + 2 * P, ct3 + 3 * P);
    to_coef(c, d2.data(), nl);
    std::vector<u64> ks(2 * P);
    u64 g = 1;
    u64* o = ks.data();
    keyswitch_hoisted(c, d2.data(), level, 1, &g, &rlk, &o);
    for (int p = 0; p < 2; p++)
        for (int i = 0; i < nl; i++) {
            const u64 q = c.mod[i];
            for (size_t x = 0; x < N; x++) {
                size_t idx = p * P + (size_t)i * N + x;
                out[idx] = add_mod(ct3[idx], ks[idx], q);
            }
        }
}

// rescale (implied by the scale-2^40 / depth-3 parameters): drop q_l with centred rounding.
static void rescale(const OrCtx& c, const u64* ct, int deg, int level, u64* out) {
    const size_t N = c.N;
    const int nl = level + 1;
    const u64 ql = c.mod[level];
    for (int p = 0; p < deg; p++) {
        const u64* in = ct + (size_t)p * nl * N;
        u64* o = out + (size_t)p * level * N;
        std::vector<u64> last(in + (size_t)level * N, in + (size_t)nl * N);
        ntt_inv(c, level, last.data());
#pragma omp parallel for schedule(static) if (!omp_in_parallel())
        for (int i = 0; i < level; i++) {
            const u64 qi = c.mod[i];
            const u64 ql_inv = inv_mod(ql % qi, qi);
            std::vector<u64> r(N);
            for (size_t x = 0; x < N; x++) {
                i64 cr = last[x] <= (ql - 1) / 2 ? (i64)last[x] : (i64)last[x] - (i64)ql;
                r[x] = from_signed(cr, qi);
            }
            ntt_fwd(c, i, r.data());
            for (size_t x = 0; x < N; x++)
                o[(size_t)i * N + x] = mul_mod(sub_mod(in[(size_t)i * N + x], r[x], qi), ql_inv, qi);
        }
    }
}

// rotation of ct by several Galois elements from one ModUp of c1 (hoisted; Section
// "Dynamic Hoisting"): out_r = (phi_g(c0) + KS_0, KS_1).
static void rotate_hoisted(OrCtx& c, const u64* ct, int level, int n_rot, const u64* gs,
                           const u64* const* keys, u64* const* outs) {
    const size_t N = c.N;
    const int nl = level + 1;
    const size_t P = (size_t)nl * N;
    std::vector<u64> c0(ct, ct + P), c1(ct + P, ct + 2 * P);
    to_coef(c, c0.data(), nl);
    to_coef(c, c1.data(), nl);
    keyswitch_hoisted(c, c1.data(), level, n_rot, gs, keys, outs);
    for (int r = 0; r < n_rot; r++) {
        std::vector<u64> a0(P);
        for (int i = 0; i < nl; i++) automorph_row(c, c0.data() + (size_t)i * N, a0.data() + (size_t)i * N, c.mod[i], gs[r]);
        to_eval(c, a0.data(), nl);
        for (int i = 0; i < nl; i++)
            for (size_t x = 0; x < N; x++)
                outs[r][(size_t)i * N + x] = add_mod(outs[r][(size_t)i * N + x], a0[(size_t)i * N + x], c.mod[i]);
    }
}

// Hoisted group with the inner products summed in Q_l U P (one ModDown for the whole group):
// out = (sum_r phi_{g_r}(c0) + ModDown(sum_r u0_r), ModDown(sum_r u1_r)).
static void rotate_group_qpsum(OrCtx& c, const u64* ct, int level, int n_rot, const u64* gs,
                               const u64* const* keys, u64* out) {
    const size_t N = c.N;
    const int nl = level + 1;
    const size_t P = (size_t)nl * N;
    std::vector<u64> c0(ct, ct + P), c1(ct + P, ct + 2 * P);
    to_coef(c, c0.data(), nl);
    to_coef(c, c1.data(), nl);
    std::vector<u64*> outs(n_rot, out);
    keyswitch_hoisted(c, c1.data(), level, n_rot, gs, keys, outs.data(), true);
    for (int r = 0; r < n_rot; r++) {
        std::vector<u64> a0(P);
        for (int i = 0; i < nl; i++) automorph_row(c, c0.data() + (size_t)i * N, a0.data() + (size_t)i * N, c.mod[i], gs[r]);
        to_eval(c, a0.data(), nl);
        for (int i = 0; i < nl; i++)
            for (size_t x = 0; x < N; x++)
                out[(size_t)i * N + x] = add_mod(out[(size_t)i * N + x], a0[(size_t)i * N + x], c.mod[i]);
    }
}

static u64 galois_of_rotation(const OrCtx& c, long r) { return pow_mod(5, (u64)r, 2 * (u64)c.N); }

// rotate-and-sum with a hoisting schedule: for each group of size g (stride s, starting at 1):
// y <- y + sum_{t=1}^{2^g-1} Rot_{t s}(y), all from one ModUp of y; then s <- s 2^g.
static int rotate_sum(OrCtx& c, u64* ct, int level, int n_groups, const int* groups,
                      int n_keys, const int* key_rot, const u64* const* keys, bool qp_sum = false) {
    const size_t P = (size_t)(level + 1) * c.N;
    long stride = 1;
    for (int gi = 0; gi < n_groups; gi++) {
        const int cnt = (1 << groups[gi]) - 1;
        std::vector<u64> gs(cnt);
        std::vector<const u64*> ks(cnt);
        std::vector<std::vector<u64>> outs(cnt, std::vector<u64>(2 * P));
        std::vector<u64*> op(cnt);
        for (int t = 1; t <= cnt; t++) {
            long r = (long)t * stride;
            gs[t - 1] = galois_of_rotation(c, r);
            ks[t - 1] = nullptr;
            for (int k = 0; k < n_keys; k++)
                if (key_rot[k] == r) ks[t - 1] = keys[k];
            if (!ks[t - 1]) return -1;
            op[t - 1] = outs[t - 1].data();
        }
        int nsum = cnt;
        if (qp_sum) {
            rotate_group_qpsum(c, ct, level, cnt, gs.data(), ks.data(), op[0]);
            nsum = 1;
        } else {
            rotate_hoisted(c, ct, level, cnt, gs.data(), ks.data(), op.data());
        }
        for (int t = 0; t < nsum; t++)
            for (int p = 0; p < 2; p++)
                for (int i = 0; i <= level; i++)
                    for (size_t x = 0; x < c.N; x++) {
                        size_t idx = p * P + (size_t)i * c.N + x;
                        ct[idx] = add_mod(ct[idx], outs[t][idx], c.mod[i]);
                    }
        stride <<= groups[gi];
    }
    return 0;
}

// ------------------------------------------------------------------ C API
// ---------------------------------------------------------------------------------------
// Device-randomness mode: the counter-based generator Philox4x64-10 (Salmon, Moraes, Dror,
// Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC 2011), written from its definition:
// ten rounds of two 64x64 -> 128-bit multiplications and a Weyl-sequence key schedule.
// Sampling rules (shared by definition with the library, not by code):
//   key = (seed, 0); counter = (coefficient k, ciphertext index c, purpose p, 0), p = 0 for the
//   ephemeral r, 1 for e0, 2 for e1; one block of four words per (k, c, p);
//   r = floor(3 * (word0 >> 32) / 2^32) - 1  in {-1, 0, 1};
//   e = popcount(word0 mod 2^21) - popcount(word1 mod 2^21)  (centred binomial, eta = 21).
static void philox4x64_10(const u64 ctr[4], const u64 key[2], u64 out[4]) {
    const u64 M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const u64 W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
    u64 x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3], k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        if (r) {
            k0 += W0;
            k1 += W1;
        }
        const u128 p0 = (u128)M0 * x0, p1 = (u128)M1 * x2;
        const u64 hi0 = (u64)(p0 >> 64), lo0 = (u64)p0, hi1 = (u64)(p1 >> 64), lo1 = (u64)p1;
        const u64 y0 = hi1 ^ x1 ^ k0, y2 = hi0 ^ x3 ^ k1;
        x0 = y0;
        x1 = lo1;
        x2 = y2;
        x3 = lo0;
    }
    out[0] = x0;
    out[1] = x1;
    out[2] = x2;
    out[3] = x3;
}

static int popcount64(u64 v) {
    int n = 0;
    for (; v; v &= v - 1) n++;
    return n;
}

extern "C" {

void or_philox4x64(const u64* ctr, const u64* key, u64* out) { philox4x64_10(ctr, key, out); }

// encryption randomness of ciphertexts first .. first+count-1 (rows of n coefficients)
void or_sample_enc(u64 seed, u64 first, int count, int n, int8_t* r, int32_t* e0, int32_t* e1) {
    const u64 key[2] = {seed, 0};
    const u64 m21 = (1ull << 21) - 1;
    for (int b = 0; b < count; b++)
        for (int k = 0; k < n; k++) {
            u64 o[4];
            const size_t i = (size_t)b * n + k;
            u64 ctr[4] = {(u64)k, first + (u64)b, 0, 0};
            philox4x64_10(ctr, key, o);
            r[i] = (int8_t)((int)(((o[0] >> 32) * 3) >> 32) - 1);
            ctr[2] = 1;
            philox4x64_10(ctr, key, o);
            e0[i] = popcount64(o[0] & m21) - popcount64(o[1] & m21);
            ctr[2] = 2;
            philox4x64_10(ctr, key, o);
            e1[i] = popcount64(o[0] & m21) - popcount64(o[1] & m21);
        }
}

int or_gen_primes(int log_n, int bits, int skip, int count, u64* out) {
    const u64 M = (u64)2 << log_n;  // 2N
    const u64 top = (bits == 64) ? ~(u64)0 : (((u64)1 << bits) - 1);
    const u64 floor_ = (u64)1 << (bits - 1);
    u64 cnd = (top / M) * M + 1;
    if (cnd > top) cnd -= M;
    int found = 0;
    while (found < skip + count) {
        if (cnd < floor_ || cnd <= M) return -1;
        if (is_prime(cnd)) {
            if (found >= skip) out[found - skip] = cnd;
            found++;
        }
        cnd -= M;
    }
    return 0;
}

OrCtx* or_ctx_new(int log_n, int nq, int np, int dnum, const u64* q, const u64* p) {
    OrCtx* c = new OrCtx();
    c->logN = log_n;
    c->N = (size_t)1 << log_n;
    c->nq = nq;
    c->np = np;
    c->dnum = dnum;
    c->alpha = (nq + dnum - 1) / dnum;  // alpha = ceil((L+1)/dnum)
    for (int i = 0; i < nq; i++) c->mod.push_back(q[i]);
    for (int i = 0; i < np; i++) c->mod.push_back(p[i]);
    const size_t N = c->N;
    c->bitrev.resize(N);
    for (size_t i = 0; i < N; i++) {
        size_t r = 0;
        for (int b = 0; b < log_n; b++)
            if (i >> b & 1) r |= (size_t)1 << (log_n - 1 - b);
        c->bitrev[i] = r;
    }
    const int nm = nq + np;
    c->psi.resize(nm);
    c->n_inv.resize(nm);
    c->psi_pow.resize(nm);
    c->psi_inv_pow.resize(nm);
    c->om_pow.resize(nm);
    c->om_inv_pow.resize(nm);
    for (int m = 0; m < nm; m++) {
        const u64 qm = c->mod[m];
        u64 psi = 0;
        for (u64 x = 2; x < qm; x++) {
            u64 w = pow_mod(x, (qm - 1) / (2 * N), qm);
            if (pow_mod(w, N, qm) == qm - 1) { psi = w; break; }
        }
        c->psi[m] = psi;
        const u64 psi_inv = inv_mod(psi, qm), om = mul_mod(psi, psi, qm), om_inv = inv_mod(om, qm);
        c->n_inv[m] = inv_mod(N % qm, qm);
        c->psi_pow[m].resize(N);
        c->psi_inv_pow[m].resize(N);
        c->om_pow[m].resize(N / 2);
        c->om_inv_pow[m].resize(N / 2);
        u64 a = 1, b = 1;
        for (size_t i = 0; i < N; i++) {
            c->psi_pow[m][i] = a;
            c->psi_inv_pow[m][i] = b;
            a = mul_mod(a, psi, qm);
            b = mul_mod(b, psi_inv, qm);
        }
        a = 1; b = 1;
        for (size_t i = 0; i < N / 2; i++) {
            c->om_pow[m][i] = a;
            c->om_inv_pow[m][i] = b;
            a = mul_mod(a, om, qm);
            b = mul_mod(b, om_inv, qm);
        }
    }
    return c;
}

void or_ctx_free(OrCtx* c) { delete c; }
int or_alpha(const OrCtx* c) { return c->alpha; }
u64 or_psi(const OrCtx* c, int mi) { return c->psi[mi]; }
void or_counters(const OrCtx* c, long long* out) { out[0] = c->n_keyswitch; out[1] = c->n_modup; }
void or_reset_counters(OrCtx* c) { c->n_keyswitch = 0; c->n_modup = 0; }
int or_set_threads(int n) { if (n > 0) omp_set_num_threads(n); return omp_get_max_threads(); }

void or_ntt_fwd(const OrCtx* c, int mi, u64* a) { ntt_fwd(*c, mi, a); }
void or_ntt_inv(const OrCtx* c, int mi, u64* a) { ntt_inv(*c, mi, a); }

// polynomials with rows q_0..q_{nrows-1}: domain conversion of `count` consecutive polys
void or_to_coeff(const OrCtx* c, u64* data, int count, int nrows) {
    for (int k = 0; k < count; k++) to_coef(*c, data + (size_t)k * nrows * c->N, nrows);
}
void or_to_eval(const OrCtx* c, u64* data, int count, int nrows) {
    for (int k = 0; k < count; k++) to_eval(*c, data + (size_t)k * nrows * c->N, nrows);
}
// key layout [dnum][2][nq+np][N]: conversion of every row with its own modulus
void or_key_to_coeff(const OrCtx* c, u64* key) {
    const int rows = c->nq + c->np;
    for (int j = 0; j < c->dnum; j++)
        for (int p = 0; p < 2; p++)
#pragma omp parallel for schedule(static)
            for (int t = 0; t < rows; t++) ntt_inv(*c, t, key + (((size_t)j * 2 + p) * rows + t) * c->N);
}

// negacyclic product through the transform (pinned against schoolbook convolution)
void or_poly_mul(const OrCtx* c, int mi, const u64* a, const u64* b, u64* out) {
    const size_t N = c->N;
    std::vector<u64> x(a, a + N), y(b, b + N);
    ntt_fwd(*c, mi, x.data());
    ntt_fwd(*c, mi, y.data());
    for (size_t i = 0; i < N; i++) x[i] = mul_mod(x[i], y[i], c->mod[mi]);
    ntt_inv(*c, mi, x.data());
    std::memcpy(out, x.data(), N * sizeof(u64));
}

// coefficient-domain automorphism of nrows rows (row t uses modulus index mods[t])
void or_automorph_coeff(const OrCtx* c, const u64* in, int nrows, const int* mods, u64 g, u64* out) {
    for (int t = 0; t < nrows; t++)
        automorph_row(*c, in + (size_t)t * c->N, out + (size_t)t * c->N, c->mod[mods[t]], g);
}
u64 or_galois(const OrCtx* c, long r) { return galois_of_rotation(*c, r); }

// pinning helpers in the coefficient domain
void or_modup_coeff(const OrCtx* c, const u64* c_coef, int level, int j, u64* ext) {
    modup_digit(*c, c_coef, level, j, ext);
}
void or_moddown_coeff(const OrCtx* c, const u64* u_coef, int level, u64* out) {
    moddown_coef(*c, u_coef, level, out);
}

// pk = (-a s + e, a) over Q (paper: Key generation, Public key).  a: coefficient domain
// [nq][N]; out: evaluation domain [2][nq][N].
void or_pk_gen(const OrCtx* c, const int8_t* s, const u64* a, const int32_t* e, u64* out) {
    const size_t N = c->N;
    const int nq = c->nq;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < nq; i++) {
        const u64 q = c->mod[i];
        std::vector<u64> sv(N), av(a + (size_t)i * N, a + (size_t)(i + 1) * N), ev(N);
        for (size_t x = 0; x < N; x++) { sv[x] = from_signed(s[x], q); ev[x] = from_signed(e[x], q); }
        ntt_fwd(*c, i, sv.data());
        ntt_fwd(*c, i, av.data());
        ntt_fwd(*c, i, ev.data());
        for (size_t x = 0; x < N; x++) {
            out[(size_t)i * N + x] = sub_mod(ev[x], mul_mod(av[x], sv[x], q), q);
            out[((size_t)nq + i) * N + x] = av[x];
        }
    }
}

// switching key from s~ to s (galois g = 0: s~ = s^2 for relinearisation; otherwise
// s~ = phi_g(s)).  Digit j, row t of Q U P:
//   b = -a_j s + e_j + [q_t in D_j] (P mod q_t) s~,   a = a_j.
// a: coefficient domain [dnum][nq+np][N]; e: [dnum][N]; out: evaluation [dnum][2][nq+np][N].
void or_swk_gen(const OrCtx* c, const int8_t* s, u64 g, const u64* a, const int32_t* e, u64* out) {
    const size_t N = c->N;
    const int rows = c->nq + c->np;
    std::vector<i64> s_signed(N);
    for (size_t x = 0; x < N; x++) s_signed[x] = s[x];
#pragma omp parallel for schedule(static)
    for (int t = 0; t < rows; t++) {
        const u64 m = c->mod[t];
        std::vector<u64> sv(N), st(N);
        for (size_t x = 0; x < N; x++) sv[x] = from_signed(s_signed[x], m);
        if (g == 0) {
            ntt_fwd(*c, t, sv.data());
            for (size_t x = 0; x < N; x++) st[x] = mul_mod(sv[x], sv[x], m);
        } else {
            automorph_row(*c, sv.data(), st.data(), m, g);
            ntt_fwd(*c, t, sv.data());
            ntt_fwd(*c, t, st.data());
        }
        u64 P_mod = 1 % m;
        for (int k = 0; k < c->np; k++) P_mod = mul_mod(P_mod, c->mod[c->nq + k] % m, m);
        for (int j = 0; j < c->dnum; j++) {
            std::vector<u64> av(a + ((size_t)j * rows + t) * N, a + ((size_t)j * rows + t + 1) * N), ev(N);
            for (size_t x = 0; x < N; x++) ev[x] = from_signed(e[(size_t)j * N + x], m);
            ntt_fwd(*c, t, av.data());
            ntt_fwd(*c, t, ev.data());
            const bool in_digit = t < c->nq && t >= j * c->alpha && t < (j + 1) * c->alpha;
            u64* ob = out + (((size_t)j * 2 + 0) * rows + t) * N;
            u64* oa = out + (((size_t)j * 2 + 1) * rows + t) * N;
            for (size_t x = 0; x < N; x++) {
                u64 b = sub_mod(ev[x], mul_mod(av[x], sv[x], m), m);
                if (in_digit) b = add_mod(b, mul_mod(P_mod, st[x], m), m);
                ob[x] = b;
                oa[x] = av[x];
            }
        }
    }
}

// Enc(pk, m) = (m + r u0 + e0, r u1 + e1) mod Q at level L (paper: Encryption).
// pk evaluation [2][nq][N]; m integer coefficients; out evaluation [2][nq][N].
void or_encrypt(const OrCtx* c, const u64* pk, const i64* m, const int8_t* r, const int32_t* e0,
                const int32_t* e1, u64* out) {
    const size_t N = c->N;
    const int nq = c->nq;
#pragma omp parallel for schedule(static) if (!omp_in_parallel())
    for (int i = 0; i < nq; i++) {
        const u64 q = c->mod[i];
        std::vector<u64> mv(N), rv(N), x0(N), x1(N);
        for (size_t x = 0; x < N; x++) {
            mv[x] = from_signed(m[x], q);
            rv[x] = from_signed(r[x], q);
            x0[x] = from_signed(e0[x], q);
            x1[x] = from_signed(e1[x], q);
        }
        ntt_fwd(*c, i, mv.data());
        ntt_fwd(*c, i, rv.data());
        ntt_fwd(*c, i, x0.data());
        ntt_fwd(*c, i, x1.data());
        for (size_t x = 0; x < N; x++) {
            const u64 u0 = pk[(size_t)i * N + x], u1 = pk[((size_t)nq + i) * N + x];
            out[(size_t)i * N + x] = add_mod(add_mod(mv[x], mul_mod(rv[x], u0, q), q), x0[x], q);
            out[((size_t)nq + i) * N + x] = add_mod(mul_mod(rv[x], u1, q), x1[x], q);
        }
    }
}

// Dec(sk, ct) = c0 + c1 s mod Q_l (paper: Decryption).  Output: coefficient-domain residues [l+1][N].
void or_decrypt(const OrCtx* c, const int8_t* s, const u64* ct, int deg, int level, u64* out) {
    const size_t N = c->N;
    const int nl = level + 1;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < nl; i++) {
        const u64 q = c->mod[i];
        std::vector<u64> sv(N), acc(N, 0), sp(N);
        for (size_t x = 0; x < N; x++) sv[x] = from_signed(s[x], q);
        ntt_fwd(*c, i, sv.data());
        for (size_t x = 0; x < N; x++) sp[x] = 1 % q;
        for (int p = 0; p < deg; p++) {
            const u64* cp = ct + ((size_t)p * nl + i) * N;
            for (size_t x = 0; x < N; x++) {
                acc[x] = add_mod(acc[x], mul_mod(cp[x], sp[x], q), q);
                sp[x] = mul_mod(sp[x], sv[x], q);
            }
        }
        ntt_inv(*c, i, acc.data());
        std::memcpy(out + (size_t)i * N, acc.data(), N * sizeof(u64));
    }
}

// HAdd / HSub (coefficient-wise mod q_i) on `deg` polynomials at level l
void or_add(const OrCtx* c, const u64* a, const u64* b, int deg, int level, u64* out) {
    const size_t N = c->N;
    for (int p = 0; p < deg; p++)
        for (int i = 0; i <= level; i++)
            for (size_t x = 0; x < N; x++) {
                size_t idx = ((size_t)p * (level + 1) + i) * N + x;
                out[idx] = add_mod(a[idx], b[idx], c->mod[i]);
            }
}
void or_sub(const OrCtx* c, const u64* a, const u64* b, int deg, int level, u64* out) {
    const size_t N = c->N;
    for (int p = 0; p < deg; p++)
        for (int i = 0; i <= level; i++)
            for (size_t x = 0; x < N; x++) {
                size_t idx = ((size_t)p * (level + 1) + i) * N + x;
                out[idx] = sub_mod(a[idx], b[idx], c->mod[i]);
            }
}

// CKKS.Mult tensor: (c0 c0', c0 c1' + c1 c0', c1 c1') in the evaluation domain
void or_tensor(const OrCtx* c, const u64* a, const u64* b, int level, u64* out) {
    const size_t N = c->N, P = (size_t)(level + 1) * N;
    for (int i = 0; i <= level; i++) {
        const u64 q = c->mod[i];
        for (size_t x = 0; x < N; x++) {
            size_t k = (size_t)i * N + x;
            out[k] = mul_mod(a[k], b[k], q);
            out[P + k] = add_mod(mul_mod(a[k], b[P + k], q), mul_mod(a[P + k], b[k], q), q);
            out[2 * P + k] = mul_mod(a[P + k], b[P + k], q);
        }
    }
}

void or_relin(OrCtx* c, const u64* ct3, int level, const u64* rlk, u64* out) { relin(*c, ct3, level, rlk, out); }
void or_rescale(const OrCtx* c, const u64* ct, int deg, int level, u64* out) { rescale(*c, ct, deg, level, out); }

// key switch of one evaluation-domain polynomial (pinning helper): out = KS(c) [2][l+1][N]
void or_keyswitch(OrCtx* c, const u64* poly_eval, int level, const u64* key, u64* out) {
    std::vector<u64> cc(poly_eval, poly_eval + (size_t)(level + 1) * c->N);
    to_coef(*c, cc.data(), level + 1);
    u64 g = 1;
    keyswitch_hoisted(*c, cc.data(), level, 1, &g, &key, &out);
}

// n_rot rotations of one ciphertext from a single ModUp
void or_rotate_hoisted(OrCtx* c, const u64* ct, int level, int n_rot, const long* rots,
                       const u64* const* keys, u64* const* outs) {
    std::vector<u64> gs(n_rot);
    for (int r = 0; r < n_rot; r++) gs[r] = galois_of_rotation(*c, rots[r]);
    rotate_hoisted(*c, ct, level, n_rot, gs.data(), keys, outs);
}

int or_rotate_sum(OrCtx* c, u64* ct, int level, int n_groups, const int* groups, int n_keys,
                  const int* key_rot, const u64* const* keys, int qp_sum) {
    return rotate_sum(*c, ct, level, n_groups, groups, n_keys, key_rot, keys, qp_sum != 0);
}

// Server distances (Algorithm 1, "Server Executes"): for each pair i<j (lexicographic):
//   acc = sum_k (ct_i[k] - ct_j[k])^2   (degree-2, lazy: no relinearisation inside the loop)
//   Dis = rotate_sum(rescale(relin(acc)))
// cts: evaluation domain [n][chunks][2][L+1][N]; out: [n_pairs][2][L][N].
// pair_list (optional, length 2*n_pairs_sel) restricts the work to the listed pairs, written
// to out in list order.
static int distances_at(OrCtx* c, const u64* cts, int n, int chunks, const u64* rlk, int n_groups,
                        const int* groups, int n_keys, const int* key_rot, const u64* const* keys,
                        int n_sel, const int* pair_list, int qp_sum, int rot_level, u64* out);

int or_distances(OrCtx* c, const u64* cts, int n, int chunks, const u64* rlk, int n_groups,
                 const int* groups, int n_keys, const int* key_rot, const u64* const* keys,
                 int n_sel, const int* pair_list, int qp_sum, u64* out) {
    return distances_at(c, cts, n, chunks, rlk, n_groups, groups, n_keys, key_rot, keys, n_sel, pair_list, qp_sum,
                        c->nq - 2, out);
}

// The same with the rescaled pair reduced to level rot_level before the rotate-and-sum: a level
// drop keeps the limbs q_0 .. q_rot_level and discards the others (a ciphertext mod Q is also one
// mod any Q' dividing Q, encrypting the same message while that message stays below Q'/2).
// out: [n_pairs][2][rot_level + 1][N].
int or_distances_dropped(OrCtx* c, const u64* cts, int n, int chunks, const u64* rlk, int n_groups,
                         const int* groups, int n_keys, const int* key_rot, const u64* const* keys,
                         int n_sel, const int* pair_list, int qp_sum, int rot_level, u64* out) {
    if (rot_level < 0 || rot_level > c->nq - 2) return -2;
    return distances_at(c, cts, n, chunks, rlk, n_groups, groups, n_keys, key_rot, keys, n_sel, pair_list, qp_sum,
                        rot_level, out);
}

static int distances_at(OrCtx* c, const u64* cts, int n, int chunks, const u64* rlk, int n_groups,
                        const int* groups, int n_keys, const int* key_rot, const u64* const* keys,
                        int n_sel, const int* pair_list, int qp_sum, int rot_level, u64* out) {
    const size_t N = c->N;
    const int L = c->nq - 1, nl = L + 1;
    const size_t P = (size_t)nl * N, CT = 2 * P;
    std::vector<int> pi, pj;
    if (n_sel > 0) {
        for (int k = 0; k < n_sel; k++) { pi.push_back(pair_list[2 * k]); pj.push_back(pair_list[2 * k + 1]); }
    } else {
        for (int i = 0; i < n; i++)
            for (int j = i + 1; j < n; j++) { pi.push_back(i); pj.push_back(j); }
    }
    const int np_ = (int)pi.size();
    int status = 0;
    // parallel over pairs when there are enough of them, else over limbs inside each step
#pragma omp parallel for schedule(dynamic, 1) if (np_ >= omp_get_max_threads())
    for (int k = 0; k < np_; k++) {
        std::vector<u64> acc(3 * P, 0), diff(CT), sq(3 * P);
        for (int ch = 0; ch < chunks; ch++) {
            const u64* a = cts + ((size_t)pi[k] * chunks + ch) * CT;
            const u64* b = cts + ((size_t)pj[k] * chunks + ch) * CT;
            or_sub(c, a, b, 2, L, diff.data());
            or_tensor(c, diff.data(), diff.data(), L, sq.data());
            or_add(c, acc.data(), sq.data(), 3, L, acc.data());
        }
        std::vector<u64> r2(CT), rs(2 * (size_t)L * N);
        relin(*c, acc.data(), L, rlk, r2.data());
        rescale(*c, r2.data(), 2, L, rs.data());
        // level drop: keep limbs 0 .. rot_level of both polynomials
        const size_t lo = (size_t)(rot_level + 1) * N;
        std::vector<u64> y(2 * lo);
        for (int p = 0; p < 2; p++) std::memcpy(y.data() + p * lo, rs.data() + (size_t)p * L * N, lo * sizeof(u64));
        int st = rotate_sum(*c, y.data(), rot_level, n_groups, groups, n_keys, key_rot, keys, qp_sum != 0);
        if (st) status = st;
        std::memcpy(out + (size_t)k * 2 * lo, y.data(), y.size() * sizeof(u64));
    }
    return status;
}

// ServerUpdate (Algorithm 1) with the mask folded into one ciphertext per client:
//   out[k] = rescale(relin(sum_i ct_i[k] (x) M_i)) for every chunk k.
// masks: evaluation [n][2][L+1][N]; out [chunks][2][L][N].
void or_masked_aggregate(OrCtx* c, const u64* cts, int n, int chunks, const u64* masks, const u64* rlk, u64* out) {
    const size_t N = c->N;
    const int L = c->nq - 1;
    const size_t P = (size_t)(L + 1) * N, CT = 2 * P;
#pragma omp parallel for schedule(dynamic, 1) if (chunks >= omp_get_max_threads())
    for (int k = 0; k < chunks; k++) {
        std::vector<u64> acc(3 * P, 0), prod(3 * P), r2(CT);
        for (int i = 0; i < n; i++) {
            or_tensor(c, cts + ((size_t)i * chunks + k) * CT, masks + (size_t)i * CT, L, prod.data());
            or_add(c, acc.data(), prod.data(), 3, L, acc.data());
        }
        relin(*c, acc.data(), L, rlk, r2.data());
        rescale(*c, r2.data(), 2, L, out + (size_t)k * 2 * L * N);
    }
}

}  // extern "C"

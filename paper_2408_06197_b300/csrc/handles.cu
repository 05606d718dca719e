// Handle layer of the C ABI: ciphertext arrays that carry their degree, level and scale, the
// secret and public keys of the key generation center, one-call key generation, encryption into
// handles, and the method's calls on handles with level / scale validation.  Every call is built
// on the array entry points of capi.cu (the kernels are the same); the handles add the metadata
// that lets the library reject a ciphertext at the wrong level or scale instead of computing on it.
#include <cuda_runtime.h>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>
#include "context.cuh"

namespace {

int hfail(lc_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    return code;
}

// One device allocation, shared by a handle and its views; released when the last one goes.
struct CtBuf {
    lc_ctx* ctx;
    u64* p;
    ~CtBuf() { lc_dev_free(ctx, p); }
};

}  // namespace

struct lc_ct {
    lc_ctx* ctx;
    std::shared_ptr<CtBuf> buf;
    u64* data;  // [count][deg][level+1][N], evaluation domain
    uint32_t count, deg, level;
    double scale;
};

struct lc_sk {
    lc_ctx* ctx;
    std::vector<int8_t> s;  // ternary secret, host copy (the KGC's)
};

struct lc_pk {
    lc_ctx* ctx;
    u64* data;  // [2][n_q][N], evaluation domain
};

namespace {

size_t ct_words(const lc_ctx* c, uint32_t deg, uint32_t level) { return (size_t)deg * (level + 1) * c->N; }

// allocates a handle of `count` ciphertexts (device words not initialised)
int new_ct(lc_ctx* c, uint32_t count, uint32_t deg, uint32_t level, double scale, lc_ct** out) {
    const size_t words = (size_t)count * ct_words(c, deg, level);
    u64* p = static_cast<u64*>(lc_dev_alloc(c, words ? words * 8 : 256));
    if (!p) return hfail(c, LC_ENOMEM, "ciphertext handle: device allocation failed");
    lc_ct* h = new (std::nothrow) lc_ct{c, nullptr, p, count, deg, level, scale};
    if (h) h->buf.reset(new (std::nothrow) CtBuf{c, p});
    if (!h || !h->buf) {
        delete h;
        lc_dev_free(c, p);
        return hfail(c, LC_ENOMEM, "ciphertext handle: host allocation failed");
    }
    *out = h;
    return LC_OK;
}

bool scale_ok(double s) { return s > 0.0 && std::isfinite(s); }

// Checks the clients of one evaluation: n handles of the same context, degree 2 (two
// polynomials), level L, one chunk count and one scale.  *chunks and *scale return them.
int check_clients(lc_ctx* c, const lc_ct* const* cl, uint32_t n, const char* what, uint32_t* chunks, double* scale) {
    if (!cl) return hfail(c, LC_EINVAL, std::string(what) + ": null client array");
    const uint32_t L = (uint32_t)c->nq - 1;
    for (uint32_t i = 0; i < n; i++) {
        const lc_ct* h = cl[i];
        if (!h || h->ctx != c) return hfail(c, LC_EINVAL, std::string(what) + ": client " + std::to_string(i) +
                                                               " is null or belongs to another context");
        if (h->deg != 2) return hfail(c, LC_EINVAL, std::string(what) + ": client " + std::to_string(i) +
                                                        " is not a two-polynomial ciphertext");
        if (h->level != L)
            return hfail(c, LC_ELEVEL, std::string(what) + ": client " + std::to_string(i) + " is at level " +
                                           std::to_string(h->level) + ", the evaluation needs level " + std::to_string(L));
        if (!scale_ok(h->scale))
            return hfail(c, LC_ESCALE, std::string(what) + ": client " + std::to_string(i) + " has no valid scale");
        if (h->count != cl[0]->count || h->count == 0)
            return hfail(c, LC_EINVAL, std::string(what) + ": clients hold different (or no) chunk counts");
        if (h->scale != cl[0]->scale)
            return hfail(c, LC_ESCALE, std::string(what) + ": client " + std::to_string(i) + " has scale " +
                                           std::to_string(h->scale) + ", client 0 has " + std::to_string(cl[0]->scale));
    }
    *chunks = cl[0]->count;
    *scale = cl[0]->scale;
    return LC_OK;
}

// Masks: n handles of one ciphertext each, degree 2, level L, one scale.
int check_masks(lc_ctx* c, const lc_ct* const* m, uint32_t n, const char* what, double* scale) {
    if (!m) return hfail(c, LC_EINVAL, std::string(what) + ": null mask array");
    const uint32_t L = (uint32_t)c->nq - 1;
    for (uint32_t i = 0; i < n; i++) {
        const lc_ct* h = m[i];
        if (!h || h->ctx != c || h->deg != 2 || h->count != 1)
            return hfail(c, LC_EINVAL, std::string(what) + ": mask " + std::to_string(i) +
                                           " must be one two-polynomial ciphertext of this context");
        if (h->level != L)
            return hfail(c, LC_ELEVEL, std::string(what) + ": mask " + std::to_string(i) + " is at level " +
                                           std::to_string(h->level) + ", the evaluation needs level " + std::to_string(L));
        if (!scale_ok(h->scale) || h->scale != m[0]->scale)
            return hfail(c, LC_ESCALE, std::string(what) + ": masks must share one finite positive scale");
    }
    *scale = m[0]->scale;
    return LC_OK;
}

// Device words of n handles laid out back to back.  When the handles already are (views of one
// allocation in order) their memory is used as it is; otherwise they are gathered, with one
// device-to-device copy per handle on the context's stream, into `dst` (which the caller sized).
const u64* contiguous(lc_ctx* c, const lc_ct* const* h, uint32_t n, size_t words_each, u64* dst, int* st) {
    bool ok = true;
    for (uint32_t i = 1; i < n && ok; i++) ok = h[i]->data == h[0]->data + (size_t)i * words_each;
    if (ok) return h[0]->data;
    for (uint32_t i = 0; i < n; i++) {
        const cudaError_t e = cudaMemcpyAsync(dst + (size_t)i * words_each, h[i]->data, words_each * 8,
                                              cudaMemcpyDeviceToDevice, c->stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            *st = hfail(c, LC_ECUDA, std::string("gathering ciphertext handles: ") + cudaGetErrorString(e));
            return nullptr;
        }
    }
    return dst;
}

bool needs_gather(const lc_ct* const* h, uint32_t n, size_t words_each) {
    for (uint32_t i = 1; i < n; i++)
        if (h[i]->data != h[0]->data + (size_t)i * words_each) return true;
    return false;
}

// the context's gather buffer, grown to at least `bytes` (contents not kept)
u64* gather_buf(lc_ctx* c, size_t bytes) {
    if (bytes <= c->gather_bytes) return static_cast<u64*>(c->gather);
    cudaStreamSynchronize(c->stream);
    lc_dev_free(c, c->gather);
    c->gather = lc_dev_alloc(c, bytes);
    c->gather_bytes = c->gather ? bytes : 0;
    return static_cast<u64*>(c->gather);
}

}  // namespace

extern "C" {

// ------------------------------------------------------------------------------ ciphertext handles

int lc_ct_create(lc_ctx* c, uint32_t count, uint32_t deg, uint32_t level, double scale, lc_ct** out) {
    if (!c || !out || deg < 1 || deg > 3) return hfail(c, LC_EINVAL, "lc_ct_create: bad argument");
    if ((int)level >= c->nq) return hfail(c, LC_ELEVEL, "lc_ct_create: level out of range");
    if (!scale_ok(scale)) return hfail(c, LC_ESCALE, "lc_ct_create: scale must be finite and > 0");
    lc_ct* h = nullptr;
    const int st = new_ct(c, count, deg, level, scale, &h);
    if (st) return st;
    const size_t words = (size_t)count * ct_words(c, deg, level);
    if (words && cudaMemsetAsync(h->data, 0, words * 8, c->stream) != cudaSuccess) {
        cudaGetLastError();
        lc_ct_free(h);
        return hfail(c, LC_ECUDA, "lc_ct_create: clearing the ciphertexts failed");
    }
    *out = h;
    return LC_OK;
}

int lc_ct_import(lc_ctx* c, const uint64_t* coeffs, uint32_t count, uint32_t deg, uint32_t level, double scale,
                 lc_ct** out) {
    if (!c || !coeffs || !out || count == 0 || deg < 1 || deg > 3)
        return hfail(c, LC_EINVAL, "lc_ct_import: bad argument");
    if ((int)level >= c->nq) return hfail(c, LC_ELEVEL, "lc_ct_import: level out of range");
    if (!scale_ok(scale)) return hfail(c, LC_ESCALE, "lc_ct_import: scale must be finite and > 0");
    const size_t N = c->N;
    for (size_t b = 0; b < (size_t)count * deg; b++)
        for (uint32_t i = 0; i <= level; i++) {
            const uint64_t* row = coeffs + (b * (level + 1) + i) * N;
            const u64 q = c->mod[i];
            for (size_t x = 0; x < N; x++)
                if (row[x] >= q)
                    return hfail(c, LC_EINVAL, "lc_ct_import: residue " + std::to_string(x) + " of limb " +
                                                   std::to_string(i) + " is not below its prime");
        }
    lc_ct* h = nullptr;
    int st = new_ct(c, count, deg, level, scale, &h);
    if (st) return st;
    st = lc_memcpy_h2d(c, h->data, coeffs, (size_t)count * ct_words(c, deg, level) * 8);
    if (!st) st = lc_to_eval(c, h->data, count * deg, level);
    if (!st) st = lc_sync(c);
    if (st) {
        lc_ct_free(h);
        return st;
    }
    *out = h;
    return LC_OK;
}

int lc_ct_export(const lc_ct* h, uint64_t* coeffs, uint32_t* level, double* scale) {
    if (!h || !coeffs) return LC_EINVAL;
    lc_ctx* c = h->ctx;
    const size_t words = (size_t)h->count * ct_words(c, h->deg, h->level);
    if (words) {
        u64* t = lc_scratch(c, words * 8);
        if (!t) return hfail(c, LC_ENOMEM, "lc_ct_export: scratch");
        if (cudaMemcpyAsync(t, h->data, words * 8, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess) {
            cudaGetLastError();
            return hfail(c, LC_ECUDA, "lc_ct_export: copy failed");
        }
        int st = lc_to_coeff(c, t, h->count * h->deg, h->level);
        if (!st) st = lc_memcpy_d2h(c, coeffs, t, words * 8);
        if (!st) st = lc_sync(c);
        if (st) return st;
    }
    if (level) *level = h->level;
    if (scale) *scale = h->scale;
    return LC_OK;
}

int lc_ct_info(const lc_ct* h, uint32_t* count, uint32_t* deg, uint32_t* level, double* scale) {
    if (!h) return LC_EINVAL;
    if (count) *count = h->count;
    if (deg) *deg = h->deg;
    if (level) *level = h->level;
    if (scale) *scale = h->scale;
    return LC_OK;
}

uint64_t* lc_ct_data(const lc_ct* h) { return h ? h->data : nullptr; }

int lc_ct_view(const lc_ct* h, uint32_t first, uint32_t count, lc_ct** out) {
    if (!h || !out) return LC_EINVAL;
    if ((uint64_t)first + count > h->count || count == 0)
        return hfail(h->ctx, LC_EINVAL, "lc_ct_view: range outside the handle");
    lc_ct* v = new (std::nothrow) lc_ct{h->ctx, h->buf, h->data + (size_t)first * ct_words(h->ctx, h->deg, h->level),
                                        count, h->deg, h->level, h->scale};
    if (!v) return hfail(h->ctx, LC_ENOMEM, "lc_ct_view: host allocation failed");
    *out = v;
    return LC_OK;
}

void lc_ct_free(lc_ct* h) { delete h; }

// ------------------------------------------------------------------------------ keys

int lc_keygen(lc_ctx* c, const int8_t* s, const lc_keygen_rand* rnd, const int32_t* rot_steps, uint32_t n_rot,
              lc_sk** sk, lc_pk** pk, lc_evk** evk) {
    if (!c || !s || !rnd || (n_rot && !rot_steps) || (!sk && !pk && !evk))
        return hfail(c, LC_EINVAL, "lc_keygen: bad argument");
    if (pk && (!rnd->pk_a || !rnd->pk_e)) return hfail(c, LC_EINVAL, "lc_keygen: public-key randomness missing");
    if (evk && (!rnd->swk_a || !rnd->swk_e)) return hfail(c, LC_EINVAL, "lc_keygen: switching-key randomness missing");
    for (uint32_t k = 0; k < n_rot; k++) {
        if (rot_steps[k] < 1 || (size_t)rot_steps[k] >= c->N / 2)
            return hfail(c, LC_EINVAL, "lc_keygen: rotation steps must lie in [1, N/2)");
        for (uint32_t j = 0; j < k; j++)
            if (rot_steps[j] == rot_steps[k]) return hfail(c, LC_EINVAL, "lc_keygen: repeated rotation step");
    }
    const size_t N = c->N;
    for (size_t x = 0; x < N; x++)
        if (s[x] < -1 || s[x] > 1) return hfail(c, LC_EINVAL, "lc_keygen: the secret must be ternary");
    std::unique_ptr<lc_sk> hs;
    std::unique_ptr<lc_pk> hp;
    lc_evk* he = nullptr;
    if (sk) {
        hs.reset(new (std::nothrow) lc_sk{c, std::vector<int8_t>(s, s + N)});
        if (!hs) return hfail(c, LC_ENOMEM, "lc_keygen: host allocation failed");
    }
    if (pk) {
        u64* p = static_cast<u64*>(lc_dev_alloc(c, (size_t)2 * c->nq * N * 8));
        if (!p) return hfail(c, LC_ENOMEM, "lc_keygen: public key allocation failed");
        hp.reset(new (std::nothrow) lc_pk{c, p});
        if (!hp) {
            lc_dev_free(c, p);
            return hfail(c, LC_ENOMEM, "lc_keygen: host allocation failed");
        }
        const int st = lc_pk_gen(c, s, rnd->pk_a, rnd->pk_e, p);
        if (st) {
            lc_dev_free(c, p);
            return st;
        }
    }
    if (evk) {
        int st = lc_evk_create(c, &he);
        const size_t a_words = (size_t)c->dnum * (c->nq + c->np) * N, e_words = (size_t)c->dnum * N;
        for (uint32_t k = 0; !st && k <= n_rot; k++)
            st = lc_evk_add(c, he, s, k == 0 ? -1 : rot_steps[k - 1], rnd->swk_a + k * a_words, rnd->swk_e + k * e_words);
        if (st) {
            lc_evk_free(he);
            if (hp) lc_dev_free(c, hp->data);
            return st;
        }
    }
    const int st = lc_sync(c);
    if (st) {
        if (he) lc_evk_free(he);
        if (hp) lc_dev_free(c, hp->data);
        return st;
    }
    if (sk) *sk = hs.release();
    if (pk) *pk = hp.release();
    if (evk) *evk = he;
    return LC_OK;
}

void lc_sk_free(lc_sk* k) { delete k; }

void lc_pk_free(lc_pk* k) {
    if (!k) return;
    lc_dev_free(k->ctx, k->data);
    delete k;
}

// ------------------------------------------------------------------------------ encryption / decryption

int lc_encrypt_plain(lc_ctx* c, const lc_pk* pk, const int64_t* m, uint32_t count, double scale,
                     const lc_enc_rand* rnd, lc_ct** out) {
    if (!c || !pk || pk->ctx != c || !m || count == 0 || !rnd || !rnd->r || !rnd->e0 || !rnd->e1 || !out)
        return hfail(c, LC_EINVAL, "lc_encrypt_plain: bad argument");
    if (!scale_ok(scale)) return hfail(c, LC_ESCALE, "lc_encrypt_plain: scale must be finite and > 0");
    lc_ct* h = nullptr;
    int st = new_ct(c, count, 2, (uint32_t)c->nq - 1, scale, &h);
    if (st) return st;
    st = lc_encrypt(c, pk->data, m, rnd->r, rnd->e0, rnd->e1, count, h->data);
    if (!st) st = lc_sync(c);
    if (st) {
        lc_ct_free(h);
        return st;
    }
    *out = h;
    return LC_OK;
}

int lc_encrypt_values(lc_ctx* c, const lc_pk* pk, const double* values, size_t len, double scale,
                      const lc_enc_rand* rnd, lc_ct** out) {
    if (!c || !pk || pk->ctx != c || !values || len == 0 || !rnd || !out)
        return hfail(c, LC_EINVAL, "lc_encrypt_values: bad argument");
    if (!scale_ok(scale)) return hfail(c, LC_ESCALE, "lc_encrypt_values: scale must be finite and > 0");
    const size_t slots = c->N / 2;
    const uint32_t count = (uint32_t)((len + slots - 1) / slots);
    std::vector<int64_t> m;
    try {
        m.resize((size_t)count * c->N);
    } catch (const std::bad_alloc&) {
        return hfail(c, LC_ENOMEM, "lc_encrypt_values: host allocation failed");
    }
    for (uint32_t b = 0; b < count; b++) {
        const size_t off = (size_t)b * slots;
        const int st = lc_encode(c, values + off, std::min(slots, len - off), scale, m.data() + (size_t)b * c->N);
        if (st) return st;
    }
    return lc_encrypt_plain(c, pk, m.data(), count, scale, rnd, out);
}

int lc_decrypt_values(lc_ctx* c, const lc_sk* sk, const lc_ct* h, double* out, size_t len) {
    if (!c || !sk || sk->ctx != c || !h || h->ctx != c || !out || h->deg < 2)
        return hfail(c, LC_EINVAL, "lc_decrypt_values: bad argument");
    const size_t N = c->N, slots = N / 2;
    const uint32_t nl = h->level + 1;
    std::vector<uint64_t> res((size_t)nl * N);
    std::vector<double> mm(N), z(slots);
    for (uint32_t b = 0; b < h->count && (size_t)b * slots < len; b++) {
        int st = lc_decrypt(c, sk->s.data(), h->data + (size_t)b * ct_words(c, h->deg, h->level), h->deg, h->level,
                            res.data());
        if (!st) st = lc_crt_to_double(c, res.data(), h->level, mm.data());
        if (!st) st = lc_decode(c, mm.data(), h->scale, z.data());
        if (st) return st;
        const size_t off = (size_t)b * slots;
        std::memcpy(out + off, z.data(), std::min(slots, len - off) * sizeof(double));
    }
    return LC_OK;
}

// ------------------------------------------------------------------------------ the method on handles

int lc_ct_distances(lc_ctx* c, const lc_evk* evk, const lc_ct* const* clients, uint32_t n, uint32_t mode,
                    uint32_t n_groups, const uint32_t* groups, lc_ct** out) {
    if (!c || !evk || evk->ctx != c || !out || n < 2) return hfail(c, LC_EINVAL, "lc_ct_distances: bad argument");
    uint32_t chunks = 0;
    double scale = 0;
    int st = check_clients(c, clients, n, "lc_ct_distances", &chunks, &scale);
    if (st) return st;
    const uint32_t L = (uint32_t)c->nq - 1;
    const size_t each = (size_t)chunks * ct_words(c, 2, L);
    u64* g = nullptr;
    if (needs_gather(clients, n, each)) {
        g = gather_buf(c, (size_t)n * each * 8);
        if (!g) return hfail(c, LC_ENOMEM, "lc_ct_distances: gather buffer");
    }
    const u64* in = contiguous(c, clients, n, each, g, &st);
    if (!in) return st;
    const uint32_t rl_code = (mode >> 8) & 255u;  // LC_ROTATE_AT_LEVEL: the outputs' level
    if (rl_code > L) return hfail(c, LC_ELEVEL, "lc_ct_distances: rotation level above the rescaled level");
    lc_ct* h = nullptr;
    st = new_ct(c, n * (n - 1) / 2, 2, rl_code ? rl_code - 1 : L - 1, 1.0, &h);
    if (st) return st;
    st = lc_distances(c, evk, in, n, chunks, scale, mode, n_groups, groups, h->data, &h->scale);
    if (st) {
        lc_ct_free(h);
        return st;
    }
    *out = h;
    return LC_OK;
}

int lc_ct_masked_aggregate(lc_ctx* c, const lc_evk* evk, const lc_ct* const* clients, uint32_t n,
                           const lc_ct* const* masks, uint32_t mode, lc_ct** out) {
    if (!c || !evk || evk->ctx != c || !out || n == 0)
        return hfail(c, LC_EINVAL, "lc_ct_masked_aggregate: bad argument");
    uint32_t chunks = 0;
    double scale = 0, mscale = 0;
    int st = check_clients(c, clients, n, "lc_ct_masked_aggregate", &chunks, &scale);
    if (!st) st = check_masks(c, masks, n, "lc_ct_masked_aggregate", &mscale);
    if (st) return st;
    const uint32_t L = (uint32_t)c->nq - 1;
    const size_t each = (size_t)chunks * ct_words(c, 2, L), mw = ct_words(c, 2, L);
    const bool gc = needs_gather(clients, n, each), gm = needs_gather(masks, n, mw);
    u64* g = nullptr;
    if (gc || gm) {
        g = gather_buf(c, ((gc ? (size_t)n * each : 0) + (gm ? (size_t)n * mw : 0)) * 8);
        if (!g) return hfail(c, LC_ENOMEM, "lc_ct_masked_aggregate: gather buffer");
    }
    const u64* in = contiguous(c, clients, n, each, g, &st);
    if (!in) return st;
    const u64* min = contiguous(c, masks, n, mw, g ? g + (gc ? (size_t)n * each : 0) : nullptr, &st);
    if (!min) return st;
    lc_ct* h = nullptr;
    st = new_ct(c, chunks, 2, L - 1, 1.0, &h);
    if (st) return st;
    st = lc_masked_aggregate(c, evk, in, n, chunks, scale, min, mscale, mode, h->data, &h->scale);
    if (st) {
        lc_ct_free(h);
        return st;
    }
    *out = h;
    return LC_OK;
}

int lc_batch_run(lc_ctx* c, lc_ct_job* jobs, uint32_t n_jobs, uint32_t flags, uint32_t n_groups,
                 const uint32_t* groups) {
    if (!c || (n_jobs && !jobs)) return hfail(c, LC_EINVAL, "lc_batch_run: bad argument");
    const uint32_t L = (uint32_t)c->nq - 1;
    std::vector<uint32_t> chunks(n_jobs);
    std::vector<double> scale(n_jobs), mscale(n_jobs);
    size_t gather_words = 0;
    for (uint32_t j = 0; j < n_jobs; j++) {
        lc_ct_job& J = jobs[j];
        J.dist = nullptr;
        J.agg = nullptr;
        if (!J.evk || J.evk->ctx != c || J.n == 0 || (J.want_dist && J.n < 2) || (!J.want_dist && !J.masks))
            return hfail(c, LC_EINVAL, "lc_batch_run: job " + std::to_string(j) + " is malformed");
        const std::string what = "lc_batch_run (job " + std::to_string(j) + ")";
        int st = check_clients(c, J.clients, J.n, what.c_str(), &chunks[j], &scale[j]);
        if (!st && J.masks) st = check_masks(c, J.masks, J.n, what.c_str(), &mscale[j]);
        if (st) return st;
        const size_t each = (size_t)chunks[j] * ct_words(c, 2, L);
        if (needs_gather(J.clients, J.n, each)) gather_words += (size_t)J.n * each;
        if (J.masks && needs_gather(J.masks, J.n, ct_words(c, 2, L))) gather_words += (size_t)J.n * ct_words(c, 2, L);
    }
    u64* g = nullptr;
    if (gather_words) {
        g = gather_buf(c, gather_words * 8);
        if (!g) return hfail(c, LC_ENOMEM, "lc_batch_run: gather buffer");
    }
    std::vector<lc_job> dj, aj;
    std::vector<lc_ct*> made;
    auto release = [&]() {
        for (lc_ct* h : made) lc_ct_free(h);
    };
    u64* cur = g;
    for (uint32_t j = 0; j < n_jobs; j++) {
        lc_ct_job& J = jobs[j];
        const size_t each = (size_t)chunks[j] * ct_words(c, 2, L), mw = ct_words(c, 2, L);
        int st = LC_OK;
        const bool gc = needs_gather(J.clients, J.n, each);
        const u64* in = contiguous(c, J.clients, J.n, each, cur, &st);
        if (!in) {
            release();
            return st;
        }
        if (gc) cur += (size_t)J.n * each;
        const u64* min = nullptr;
        if (J.masks) {
            const bool gm = needs_gather(J.masks, J.n, mw);
            min = contiguous(c, J.masks, J.n, mw, cur, &st);
            if (!min) {
                release();
                return st;
            }
            if (gm) cur += (size_t)J.n * mw;
        }
        lc_job b{J.evk, in, J.n, chunks[j], min, nullptr, nullptr};
        if (J.want_dist) {
            lc_ct* h = nullptr;
            st = new_ct(c, J.n * (J.n - 1) / 2, 2, L - 1, scale[j] * scale[j] / (double)c->mod[L], &h);
            if (st) {
                release();
                return st;
            }
            made.push_back(h);
            b.out_dist = h->data;
            dj.push_back(b);
        }
        if (J.masks) {
            lc_ct* h = nullptr;
            st = new_ct(c, chunks[j], 2, L - 1, scale[j] * mscale[j] / (double)c->mod[L], &h);
            if (st) {
                release();
                return st;
            }
            made.push_back(h);
            b.out_agg = h->data;
            b.out_dist = nullptr;
            aj.push_back(b);
        }
    }
    int st = dj.empty() ? LC_OK : lc_batch_distances(c, dj.data(), (uint32_t)dj.size(), flags, n_groups, groups);
    if (!st && !aj.empty()) st = lc_batch_aggregate(c, aj.data(), (uint32_t)aj.size());
    if (st) {
        release();
        return st;
    }
    // hand the outputs to the jobs in order
    size_t k = 0;
    for (uint32_t j = 0; j < n_jobs; j++) {
        if (jobs[j].want_dist) jobs[j].dist = made[k++];
        if (jobs[j].masks) jobs[j].agg = made[k++];
    }
    return LC_OK;
}

}  // extern "C"

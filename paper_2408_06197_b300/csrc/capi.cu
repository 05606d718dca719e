// C ABI of the Lancelot server evaluation (include/lancelot.h): context and device tables,
// key generation, encryption, decryption, and the orchestration of the evaluation kernels
// (hybrid key switching, relinearisation, rescale, hoisted rotations, distances, masked
// aggregate).
#include <cuda_runtime.h>
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <cstdlib>
#include <new>
#include <string>
#include <vector>
#include "context.cuh"
#include "host_math.hpp"
#include "ops.cuh"
#include "probe.cuh"
#include "tma.cuh"
#include "wire.cuh"

using lc::hinv;
using lc::hmul;
using lc::hpow;
using lc::shoup_of;

namespace {

int fail(lc_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    return code;
}

#define LC_CUDA(c, call)                                                                   \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) return fail((c), LC_ECUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

}  // namespace

int check_launch(lc_ctx* c, const char* what) {
    if (c && !c->debug_err.empty()) {
        std::string m = c->debug_err;
        c->debug_err.clear();
        cudaGetLastError();
        return fail(c, LC_ECUDA, std::string(what) + ": " + m);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(c, LC_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return LC_OK;
}

// An entry point reports only errors of its own launches: clear a non-sticky error left by other
// code on this thread (a sticky device fault stays and is reported by the launches).
void clear_prior_error() { cudaGetLastError(); }

namespace {

RowMap rows_seq(int n, int mod0 = 0, int row0 = 0) {
    RowMap m{};
    m.n = n;
    for (int i = 0; i < n; i++) {
        m.row[i] = (uint16_t)(row0 + i);
        m.mod[i] = (uint8_t)(mod0 + i);
    }
    return m;
}

bool is_host_ptr(const void* p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
}

}  // namespace

// ------------------------------------------------------------------------------------ profiling
static void prof_begin(lc_ctx* c) {
    if (!c->prof_on || c->capturing) return;
    if (c->ev_used + 2 > c->ev_pool.size()) {
        for (int i = 0; i < 256; i++) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            c->ev_pool.push_back(e);
        }
    }
    cudaEventRecord(c->ev_pool[c->ev_used], c->stream);
}
static void prof_end(lc_ctx* c, int cls, double bytes, uint64_t units) {
    if (!c->prof_on || c->capturing) return;
    cudaEvent_t a = c->ev_pool[c->ev_used], b = c->ev_pool[c->ev_used + 1];
    cudaEventRecord(b, c->stream);
    c->ev_used += 2;
    c->prof.push_back(ProfRec{cls, a, b, bytes, units});
}
static void debug_check(lc_ctx* c, const char* what, int line) {
    if (!c->debug || !c->debug_err.empty()) return;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) c->debug_err = std::string(what) + " (capi.cu:" + std::to_string(line) + "): " + cudaGetErrorString(e);
}
#define PROF(c, cls, bytes, units, stmt)      \
    do {                                      \
        prof_begin(c);                        \
        stmt;                                 \
        prof_end(c, cls, bytes, units);       \
        debug_check(c, #stmt, __LINE__);      \
    } while (0)

// ------------------------------------------------------------------------------------ memory
void* lc_dev_alloc(lc_ctx* c, size_t bytes) {
    if (bytes == 0) bytes = 256;
    if (c->has_alloc) {
        void* p = c->alloc.alloc(bytes, c->alloc.user);
        cudaGetLastError();  // a non-sticky error raised inside the caller's allocator is not ours
        return p;
    }
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void lc_dev_free(lc_ctx* c, void* p) {
    if (!p) return;
    if (c->has_alloc) {
        c->alloc.free(p, c->alloc.user);
        cudaGetLastError();
    } else {
        cudaFree(p);
    }
}

u64* lc_scratch(lc_ctx* c, size_t bytes) {
    if (bytes <= c->scratch_bytes) return static_cast<u64*>(c->scratch);
    if (c->capturing) {
        c->err = "scratch would grow during graph capture: run the same call once before capturing";
        return nullptr;
    }
    cudaStreamSynchronize(c->stream);
    lc_dev_free(c, c->scratch);
    c->scratch = nullptr;
    c->scratch_bytes = 0;
    size_t want = bytes + bytes / 8;
    c->scratch = lc_dev_alloc(c, want);
    if (!c->scratch) return nullptr;
    c->scratch_bytes = want;
    return static_cast<u64*>(c->scratch);
}

static u64* stage_buf(lc_ctx* c, size_t bytes) {
    if (bytes <= c->stage_bytes) return static_cast<u64*>(c->stage);
    if (c->capturing) return nullptr;
    cudaStreamSynchronize(c->stream);
    lc_dev_free(c, c->stage);
    c->stage = lc_dev_alloc(c, bytes);
    c->stage_bytes = c->stage ? bytes : 0;
    return static_cast<u64*>(c->stage);
}

// ------------------------------------------------------------------------------------ tables
static int build_tables(lc_ctx* c) {
    const int nm = c->nq + c->np;
    const size_t N = c->N;
    std::vector<ulonglong2> fwd(nm * N), inv(nm * N);
    c->mc_host.resize(nm);
    std::vector<u64> pw(N), pwi(N);
    for (int m = 0; m < nm; m++) {
        const u64 q = c->mod[m];
        const u64 psi = lc::root_2n(q, c->log_n), psi_inv = hinv(psi, q);
        pw[0] = 1;
        pwi[0] = 1;
        for (size_t i = 1; i < N; i++) {
            pw[i] = hmul(pw[i - 1], psi, q);
            pwi[i] = hmul(pwi[i - 1], psi_inv, q);
        }
        const u64 ninv = hinv(N % q, q);
        for (size_t k = 0; k < N; k++) {
            const unsigned r = lc::bit_reverse((unsigned)k, c->log_n);
            fwd[m * N + k] = make_ulonglong2(pw[r], shoup_of(pw[r], q));
            inv[m * N + k] = make_ulonglong2(pwi[r], shoup_of(pwi[r], q));
        }
        const u64 last = hmul(pwi[lc::bit_reverse(1, c->log_n)], ninv, q);
        inv[m * N + 0] = make_ulonglong2(last, shoup_of(last, q));
        // entries [N / 2^(b+1), N / 2^b) serve only the row-pass stages b = 0, 1, 2 (the last
        // three forward stages, the first three inverse ones); store each group of 16 * s entries
        // (s = 2^(3-b), one group per 256-word block) lane-interleaved: entry lo * s + v at
        // v * 16 + lo (the device's tw_row_slot)
        for (int b = 0; b < 3; b++) {
            const size_t base = N >> (b + 1), s = (size_t)8 >> b, grp = 16 * s;
            for (ulonglong2* t : {&fwd[m * N], &inv[m * N]}) {
                std::vector<ulonglong2> g(grp);
                for (size_t g0 = base; g0 < 2 * base; g0 += grp) {
                    for (size_t lo = 0; lo < 16; lo++)
                        for (size_t v = 0; v < s; v++) g[v * 16 + lo] = t[g0 + lo * s + v];
                    std::copy(g.begin(), g.end(), t + g0);
                }
            }
        }
        ModConst& mc = c->mc_host[m];
        mc.q = q;
        mc.two_q = 2 * q;
        mc.r64 = (u64)(((lc::u128)1 << 64) % q);
        mc.r64_sh = shoup_of(mc.r64, q);
        mc.one_sh = (u64)(((lc::u128)1 << 64) / q);
        mc.n_inv = ninv;
        mc.n_inv_sh = shoup_of(ninv, q);
        {
            int b = 0;
            while (b < 64 && (q >> b)) b++;
            const int s1 = std::max(0, b - 25), sh = b + 31 - s1;
            const u64 cc = (b + 31 < 128) ? (u64)(((lc::u128)1 << (b + 31)) / q) : 0;
            mc.lzr = (b <= 46 && cc < (1ull << 32)) ? (cc | (u64)s1 << 32 | (u64)sh << 40) : 0;
        }
    }
    // ModUp tables [level][digit]
    std::vector<ModUpTab> mu((size_t)c->nq * c->dnum);
    for (int level = 0; level < c->nq; level++) {
        const int nl = level + 1, rows = nl + c->np;
        for (int j = 0; j < c->digits(level); j++) {
            ModUpTab& t = mu[(size_t)level * c->dnum + j];
            std::memset(&t, 0, sizeof(t));
            const int lo = j * c->alpha, hi = std::min((j + 1) * c->alpha, nl);
            t.n_src = hi - lo;
            for (int i = lo; i < hi; i++) {
                const u64 qi = c->mod[i];
                u64 prod = 1 % qi;
                for (int k = lo; k < hi; k++)
                    if (k != i) prod = hmul(prod, c->mod[k] % qi, qi);
                const int s = i - lo;
                t.src_row[s] = i;
                t.src_q[s] = qi;
                t.hinv[s] = hinv(prod, qi);
                t.hinv_sh[s] = shoup_of(t.hinv[s], qi);
            }
            int nd = 0;
            for (int r = 0; r < rows; r++) {
                if (r >= lo && r < hi) continue;
                const int mi = c->qp_mod(level, r);
                const u64 mt = c->mod[mi];
                t.dst_row[nd] = r;
                t.dst_mod[nd] = mi;
                t.dq[nd] = c->mc_host[mi].q;
                t.dr64[nd] = c->mc_host[mi].r64;
                t.dr64sh[nd] = c->mc_host[mi].r64_sh;
                t.donesh[nd] = c->mc_host[mi].one_sh;
                for (int i = lo; i < hi; i++) {
                    u64 prod = 1 % mt;
                    for (int k = lo; k < hi; k++)
                        if (k != i) prod = hmul(prod, c->mod[k] % mt, mt);
                    const int s = i - lo;
                    t.hat[s][nd] = prod;
                    const u64 qh = hmul(c->mod[i] % mt, prod, mt);
                    t.corr[s][nd] = qh ? mt - qh : 0;
                }
                nd++;
            }
            t.n_dst = nd;
        }
    }
    // ModDown table
    ModDownTab md;
    std::memset(&md, 0, sizeof(md));
    md.K = c->np;
    for (int k = 0; k < c->np; k++) {
        const u64 pk = c->mod[c->nq + k];
        u64 prod = 1 % pk;
        for (int m = 0; m < c->np; m++)
            if (m != k) prod = hmul(prod, c->mod[c->nq + m] % pk, pk);
        md.p[k] = pk;
        md.phinv[k] = hinv(prod, pk);
        md.phinv_sh[k] = shoup_of(md.phinv[k], pk);
        for (int i = 0; i < c->nq; i++) {
            const u64 qi = c->mod[i];
            u64 ph = 1 % qi;
            for (int m = 0; m < c->np; m++)
                if (m != k) ph = hmul(ph, c->mod[c->nq + m] % qi, qi);
            md.phat[k][i] = ph;
            const u64 v = hmul(pk % qi, ph, qi);
            md.corr[k][i] = v ? qi - v : 0;
        }
    }
    for (int i = 0; i < c->nq; i++) {
        const u64 qi = c->mod[i];
        u64 P = 1 % qi;
        for (int k = 0; k < c->np; k++) P = hmul(P, c->mod[c->nq + k] % qi, qi);
        md.pinv[i] = hinv(P, qi);
        md.pinv_sh[i] = shoup_of(md.pinv[i], qi);
        md.qq[i] = c->mc_host[i].q;
        md.qr64[i] = c->mc_host[i].r64;
        md.qr64sh[i] = c->mc_host[i].r64_sh;
        md.qonesh[i] = c->mc_host[i].one_sh;
    }
    // rescale tables
    std::vector<RescaleTab> rs(c->nq);
    for (int level = 0; level < c->nq; level++) {
        RescaleTab& t = rs[level];
        std::memset(&t, 0, sizeof(t));
        const u64 ql = c->mod[level];
        for (int i = 0; i < level; i++) {
            const u64 qi = c->mod[i];
            t.qinv[i] = hinv(ql % qi, qi);
            t.qinv_sh[i] = shoup_of(t.qinv[i], qi);
            const u64 r = ql % qi;
            t.negq[i] = r ? qi - r : 0;
        }
    }
    c->tw_fwd = static_cast<ulonglong2*>(lc_dev_alloc(c, fwd.size() * sizeof(ulonglong2)));
    c->tw_inv = static_cast<ulonglong2*>(lc_dev_alloc(c, inv.size() * sizeof(ulonglong2)));
    c->mc = static_cast<ModConst*>(lc_dev_alloc(c, nm * sizeof(ModConst)));
    c->modup = static_cast<ModUpTab*>(lc_dev_alloc(c, mu.size() * sizeof(ModUpTab)));
    c->moddown = static_cast<ModDownTab*>(lc_dev_alloc(c, sizeof(ModDownTab)));
    c->rescale = static_cast<RescaleTab*>(lc_dev_alloc(c, rs.size() * sizeof(RescaleTab)));
    if (!c->tw_fwd || !c->tw_inv || !c->mc || !c->modup || !c->moddown || !c->rescale)
        return fail(c, LC_ENOMEM, "table allocation failed");
    LC_CUDA(c, cudaMemcpy(c->tw_fwd, fwd.data(), fwd.size() * sizeof(ulonglong2), cudaMemcpyHostToDevice));
    LC_CUDA(c, cudaMemcpy(c->tw_inv, inv.data(), inv.size() * sizeof(ulonglong2), cudaMemcpyHostToDevice));
    LC_CUDA(c, cudaMemcpy(c->mc, c->mc_host.data(), nm * sizeof(ModConst), cudaMemcpyHostToDevice));
    LC_CUDA(c, cudaMemcpy(c->modup, mu.data(), mu.size() * sizeof(ModUpTab), cudaMemcpyHostToDevice));
    LC_CUDA(c, cudaMemcpy(c->moddown, &md, sizeof(ModDownTab), cudaMemcpyHostToDevice));
    LC_CUDA(c, cudaMemcpy(c->rescale, rs.data(), rs.size() * sizeof(RescaleTab), cudaMemcpyHostToDevice));
    return LC_OK;
}

// ------------------------------------------------------------------------------------ helpers
static void ntt_fwd_p(lc_ctx* c, u64* base, size_t stride, int batch, const RowMap& m) {
    const double limbs = (double)batch * m.n;
    PROF(c, PROF_NTT, limbs * c->N * 16.0, (uint64_t)limbs,
         ntt_forward(base, stride, batch, m, c->log_n, c->tables(), c->stream, c->ntt_tune()));
    if (c->debug && c->debug_err.size()) c->debug_err += " [forward NTT batch " + std::to_string(batch) + " rows " + std::to_string(m.n) + "]";
}
static void ntt_inv_p(lc_ctx* c, u64* base, size_t stride, int batch, const RowMap& m) {
    const double limbs = (double)batch * m.n;
    PROF(c, PROF_NTT, limbs * c->N * 16.0, (uint64_t)limbs,
         ntt_inverse(base, stride, batch, m, c->log_n, c->tables(), c->stream, c->ntt_tune()));
}
static void ntt_polys(lc_ctx* c, u64* data, int n_polys, int nl, bool forward) {
    RowMap m = rows_seq(nl);
    if (forward) ntt_fwd_p(c, data, (size_t)nl * c->N, n_polys, m);
    else ntt_inv_p(c, data, (size_t)nl * c->N, n_polys, m);
}

// Scratch words needed by key switching B polynomials at `level` with `n_out` outputs kept.
static size_t ks_words(lc_ctx* c, int B, int level) {
    const size_t N = c->N;
    const int nl = level + 1, rows = nl + c->np, beta = c->digits(level);
    return (size_t)B * N * (nl + (size_t)beta * rows + 2 * rows + 2 * nl);
}

struct KsBufs {
    u64 *coef, *ext, *v, *conv;
};

static KsBufs ks_layout(lc_ctx* c, u64* base, int B, int level) {
    const size_t N = c->N;
    const int nl = level + 1, rows = nl + c->np, beta = c->digits(level);
    KsBufs k;
    k.coef = base;
    k.ext = k.coef + (size_t)B * nl * N;
    k.v = k.ext + (size_t)B * beta * rows * N;
    k.conv = k.v + (size_t)B * 2 * rows * N;
    return k;
}

// decomposition + ModUp of B polys d (evaluation domain, stride d_stride)
static void ks_modup(lc_ctx* c, const u64* d, size_t d_stride, int B, int level, const KsBufs& k) {
    const size_t N = c->N;
    const int nl = level + 1, rows = nl + c->np, beta = c->digits(level);
    cudaMemcpy2DAsync(k.coef, (size_t)nl * N * 8, d, d_stride * 8, (size_t)nl * N * 8, B, cudaMemcpyDeviceToDevice,
                      c->stream);
    ntt_polys(c, k.coef, B, nl, false);
    PROF(c, PROF_MODUP, (double)B * N * 8.0 * ((double)nl + (double)beta * rows - nl), (uint64_t)B,
         op_modup(c, k.coef, (size_t)nl * N, B, level, k.ext));
    RowMap m{};
    int n = 0;
    for (int j = 0; j < beta; j++) {
        const int lo = j * c->alpha, hi = std::min((j + 1) * c->alpha, nl);
        for (int t = 0; t < rows; t++) {
            if (t >= lo && t < hi) continue;
            m.row[n] = (uint16_t)(j * rows + t);
            m.mod[n] = (uint8_t)c->qp_mod(level, t);
            n++;
        }
    }
    m.n = n;
    ntt_fwd_p(c, k.ext, (size_t)beta * rows * N, B, m);
    c->n_modup += (uint64_t)B;
}

// inner product with one key + ModDown; W[b] = (add0 + MD(v0), add1 + MD(v1))
// inner product of the extended digits with one key: v [B][2][rows][N]
static void ks_inner(lc_ctx* c, const u64* d, size_t d_stride, int B, int level, const u64* key, const KsBufs& k,
                     u64* v) {
    const size_t N = c->N;
    const int nl = level + 1, rows = nl + c->np;
    const int beta = c->digits(level);
    PROF(c, PROF_INNER, (double)N * 8.0 * ((double)B * beta * rows + 2.0 * beta * rows + 2.0 * B * rows), (uint64_t)B,
         op_inner(c, k.ext, d, d_stride, B, level, key, v));
    c->n_keyswitch += (uint64_t)B;
}

// ModDown of v (overwritten): W[b] = (add0 + MD(v0), add1 + MD(v1))
static void ks_moddown(lc_ctx* c, u64* v, int B, int level, const KsBufs& k, const u64* add0, size_t add0_stride,
                       const u64* add1, size_t add1_stride, u64* w, size_t w_stride) {
    const size_t N = c->N;
    const int nl = level + 1, rows = nl + c->np;
    RowMap mp{};
    mp.n = 2 * c->np;
    for (int p = 0; p < 2; p++)
        for (int m = 0; m < c->np; m++) {
            mp.row[p * c->np + m] = (uint16_t)(p * rows + nl + m);
            mp.mod[p * c->np + m] = (uint8_t)(c->nq + m);
        }
    ntt_inv_p(c, v, (size_t)2 * rows * N, B, mp);
    PROF(c, PROF_MODDOWN, (double)N * 8.0 * 2.0 * B * (c->np + nl), (uint64_t)B,
         op_moddown_bconv(c, v, B, level, k.conv));
    ntt_polys(c, k.conv, 2 * B, nl, true);
    PROF(c, PROF_MODDOWN, (double)N * 8.0 * 2.0 * B * nl * (add0 ? 4.0 : 3.0), (uint64_t)B,
         op_moddown_combine(c, v, k.conv, B, level, add0, add0_stride, add1, add1_stride, w, w_stride));
}

// ModDown of v (overwritten) fused with the rescale that follows it: out[b] (level limbs) =
// rescale(add + MD(v)), bit-identical to ks_moddown then do_rescale with one forward NTT per limb
// instead of two (op_mdrs_prep / op_mdrs_combine).  Uses k.coef (free after the inner product)
// for the last limb of (add0, add1) in the coefficient domain.
static void ks_moddown_rescale(lc_ctx* c, u64* v, int B, int level, const KsBufs& k, const u64* add0,
                               size_t add0_stride, const u64* add1, size_t add1_stride, u64* out, size_t out_stride) {
    const size_t N = c->N;
    const int nl = level + 1, rows = nl + c->np;
    RowMap mi{};
    mi.n = 2 * (c->np + 1);
    for (int p = 0; p < 2; p++) {
        for (int m = 0; m < c->np; m++) {
            mi.row[p * (c->np + 1) + m] = (uint16_t)(p * rows + nl + m);
            mi.mod[p * (c->np + 1) + m] = (uint8_t)(c->nq + m);
        }
        mi.row[p * (c->np + 1) + c->np] = (uint16_t)(p * rows + level);
        mi.mod[p * (c->np + 1) + c->np] = (uint8_t)level;
    }
    ntt_inv_p(c, v, (size_t)2 * rows * N, B, mi);
    u64* al = k.coef;  // [B][2][N]
    cudaMemcpy2DAsync(al, 2 * N * 8, add0 + (size_t)level * N, add0_stride * 8, N * 8, B, cudaMemcpyDeviceToDevice,
                      c->stream);
    cudaMemcpy2DAsync(al + N, 2 * N * 8, add1 + (size_t)level * N, add1_stride * 8, N * 8, B,
                      cudaMemcpyDeviceToDevice, c->stream);
    ntt_inv_p(c, al, N, 2 * B, rows_seq(1, level));
    PROF(c, PROF_MODDOWN, (double)N * 8.0 * 2.0 * B * (c->np + nl), (uint64_t)B,
         op_moddown_bconv(c, v, B, level, k.conv));
    PROF(c, PROF_RESCALE, (double)N * 8.0 * 2.0 * B * (2.0 * level + 3.0), (uint64_t)B,
         op_mdrs_prep(c, v, al, k.conv, B, level));
    ntt_fwd_p(c, k.conv, (size_t)nl * N, 2 * B, rows_seq(level));
    PROF(c, PROF_MODDOWN, (double)N * 8.0 * 2.0 * B * level * 4.0, (uint64_t)B,
         op_mdrs_combine(c, v, k.conv, B, level, add0, add0_stride, add1, add1_stride, out, out_stride));
}

// inner product with one key + ModDown; W[b] = (add0 + MD(v0), add1 + MD(v1))
static void ks_apply(lc_ctx* c, const u64* d, size_t d_stride, int B, int level, const u64* key, const KsBufs& k,
                     const u64* add0, const u64* add1, size_t add_stride, u64* w, size_t w_stride) {
    ks_inner(c, d, d_stride, B, level, key, k, k.v);
    ks_moddown(c, k.v, B, level, k, add0, add_stride, add1, add_stride, w, w_stride);
}

static const SwKey* find_key(const lc_evk* evk, int32_t id) {
    auto it = evk->keys.find(id);
    return it == evk->keys.end() ? nullptr : &it->second;
}

// A key set made on another context may be used when that context has the same device, ring
// degree and moduli (its keys are plain device arrays in the same layout).
static bool evk_usable(const lc_ctx* c, const lc_evk* evk) {
    const lc_ctx* o = evk ? evk->ctx : nullptr;
    return o && (o == c || (o->device == c->device && o->log_n == c->log_n && o->nq == c->nq && o->np == c->np &&
                            o->dnum == c->dnum && o->mod == c->mod));
}

// relinearise B triples ct3 [B][3][nl][N] into out [B][2][nl][N] (tmp = ks scratch)
static int do_relin(lc_ctx* c, const lc_evk* evk, const u64* ct3, int B, int level, u64* out, u64* tmp) {
    const SwKey* k = find_key(evk, -1);
    if (!k) return fail(c, LC_EKEY, "relinearisation key missing");
    const size_t P = (size_t)(level + 1) * c->N;
    KsBufs kb = ks_layout(c, tmp, B, level);
    ks_modup(c, ct3 + 2 * P, 3 * P, B, level, kb);
    ks_apply(c, ct3 + 2 * P, 3 * P, B, level, k->data, kb, ct3, ct3 + P, 3 * P, out, 2 * P);
    return LC_OK;
}

// relinearise B triples ct3 [B][3][nl][N] and rescale: out [B][2][level][N] (tmp = ks scratch)
static int do_relin_rescale(lc_ctx* c, const lc_evk* evk, const u64* ct3, int B, int level, u64* out, u64* tmp) {
    const SwKey* k = find_key(evk, -1);
    if (!k) return fail(c, LC_EKEY, "relinearisation key missing");
    const size_t P = (size_t)(level + 1) * c->N;
    KsBufs kb = ks_layout(c, tmp, B, level);
    ks_modup(c, ct3 + 2 * P, 3 * P, B, level, kb);
    ks_inner(c, ct3 + 2 * P, 3 * P, B, level, k->data, kb, kb.v);
    ks_moddown_rescale(c, kb.v, B, level, kb, ct3, 3 * P, ct3 + P, 3 * P, out, (size_t)2 * level * c->N);
    return LC_OK;
}

size_t rescale_words(lc_ctx* c, int B, int deg, int level) {
    return (size_t)B * deg * c->N * (1 + level);
}

// rescale B ciphertexts [B][deg][level+1][N] -> out [B][deg][level][N]
void do_rescale(lc_ctx* c, const u64* ct, int B, int deg, int level, u64* out, u64* tmp) {
    const size_t N = c->N;
    u64* lastc = tmp;
    u64* r = tmp + (size_t)B * deg * N;
    cudaMemcpy2DAsync(lastc, N * 8, ct + (size_t)level * N, (size_t)(level + 1) * N * 8, N * 8, (size_t)B * deg,
                      cudaMemcpyDeviceToDevice, c->stream);
    RowMap one = rows_seq(1, level);
    ntt_inv_p(c, lastc, N, B * deg, one);
    PROF(c, PROF_RESCALE, (double)N * 8.0 * B * deg * (1.0 + level), (uint64_t)B,
         op_rescale_prep(c, lastc, B * deg, level, r));
    ntt_polys(c, r, B * deg, level, true);
    PROF(c, PROF_RESCALE, (double)N * 8.0 * B * deg * (3.0 * level), (uint64_t)B,
         op_rescale_combine(c, ct, r, B, deg, level, out));
}

// algorithmic bytes of one fused group inner product: the extended digits (own rows from the
// input), the group's keys, phi(c0)'s input, and the two outputs
static double inner_gather_bytes(lc_ctx* c, int B, int level, int cnt) {
    const int nl = level + 1, rows = nl + c->np, beta = c->digits(level);
    return (double)c->N * 8.0 * ((double)B * beta * rows + 2.0 * cnt * beta * rows + 2.0 * B * rows + 2.0 * B * nl);
}

static size_t rotsum_words(lc_ctx* c, int B, int level, int max_group, bool qp_sum = false) {
    const size_t wsz = (size_t)B * 2 * (level + 1) * c->N;
    if (qp_sum)  // the group's sum over Q_l U P + accumulated phi(c0); single-rotation groups use wsz
        return ks_words(c, B, level) + std::max(wsz, (size_t)B * c->N * (2 * (level + 1 + c->np) + (level + 1)));
    return ks_words(c, B, level) + wsz * (((size_t)1 << max_group) - 1);
}

// Rotate-and-sum of B ciphertexts y [B][2][level+1][N] in place.  With qp_sum, each hoisted
// group sums its rotations' inner products over Q_l U P and switches down once:
// y <- (y0 + sum_t phi_t(y0) + MD(sum_t u0_t), y1 + MD(sum_t u1_t)), u_t = phi_t(v_t).
static int do_rotate_sum(lc_ctx* c, const lc_evk* evk, u64* y, int B, int level, int n_groups, const uint32_t* groups,
                         u64* tmp, bool qp_sum = false) {
    const size_t N = c->N;
    const int nl = level + 1, rows = nl + c->np;
    const size_t P = (size_t)nl * N;
    KsBufs kb = ks_layout(c, tmp, B, level);
    u64* wbase = tmp + ks_words(c, B, level);
    long stride = 1;
    for (int gi = 0; gi < n_groups; gi++) {
        const int g = (int)(groups ? groups[gi] : 1);
        const int cnt = (1 << g) - 1;
        std::vector<const SwKey*> keys(cnt);
        for (int t = 1; t <= cnt; t++) {
            keys[t - 1] = find_key(evk, (int32_t)(t * stride));
            if (!keys[t - 1]) return fail(c, LC_EKEY, "rotation key " + std::to_string(t * stride) + " missing");
        }
        ks_modup(c, y + P, 2 * P, B, level, kb);
        if (qp_sum && cnt > 1) {  // the fused group kernel (groups of up to 4 bits: 15 rotations)
            const size_t vsz = (size_t)B * 2 * rows * N;
            u64* usum = wbase;      // [B][2][rows][N]
            u64* c0acc = usum + vsz;  // [B][nl][N]
            std::vector<const u64*> kp(cnt);
            std::vector<uint64_t> gs(cnt);
            for (int t = 0; t < cnt; t++) {
                kp[t] = keys[t]->qp;  // group-kernel layout
                gs[t] = keys[t]->galois;
            }
            PROF(c, PROF_INNER, inner_gather_bytes(c, B, level, cnt), (uint64_t)B,
                 op_inner_gather(c, kb.ext, y + P, 2 * P, y, 2 * P, B, level, kp.data(), nullptr, gs.data(), cnt, usum,
                                 c0acc));
            c->n_keyswitch += (uint64_t)B * cnt;
            ks_moddown(c, usum, B, level, kb, c0acc, P, y + P, 2 * P, y, 2 * P);
        } else {
            for (int t = 0; t < cnt; t++)
                ks_apply(c, y + P, 2 * P, B, level, keys[t]->data, kb, y, nullptr, 2 * P,
                         wbase + (size_t)t * B * 2 * P, 2 * P);
            for (int t = 0; t < cnt; t++)
                PROF(c, PROF_AUTO, (double)B * 2 * P * 8.0 * 3.0, (uint64_t)B,
                     op_gather(c, wbase + (size_t)t * B * 2 * P, y, B * 2, level + 1, keys[t]->galois, true));
        }
        stride <<= g;
    }
    return LC_OK;
}

static uint64_t galois_of(lc_ctx* c, long r) { return hpow(5, (u64)r, 2 * (u64)c->N); }

// ------------------------------------------------------------------------------------ host FP64 encode / decode
namespace {
void fft_inplace(std::vector<std::complex<double>>& a, bool inverse) {
    const size_t n = a.size();
    for (size_t i = 1, j = 0; i < n; i++) {
        size_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(a[i], a[j]);
    }
    for (size_t len = 2; len <= n; len <<= 1) {
        const double ang = 2 * M_PI / (double)len * (inverse ? 1 : -1);
        const size_t half = len / 2;
        std::vector<std::complex<double>> w(half);
        for (size_t k = 0; k < half; k++) w[k] = std::complex<double>(std::cos(ang * k), std::sin(ang * k));
        for (size_t i = 0; i < n; i += len)
            for (size_t k = 0; k < half; k++) {
                std::complex<double> u = a[i + k], v = a[i + k + half] * w[k];
                a[i + k] = u + v;
                a[i + k + half] = u - v;
            }
    }
}

// multi-word unsigned integer (little-endian 64-bit words)
struct Big {
    std::vector<u64> w;
    void mul_add(u64 m, u64 add) {
        lc::u128 carry = add;
        for (auto& x : w) {
            lc::u128 t = (lc::u128)x * m + carry;
            x = (u64)t;
            carry = t >> 64;
        }
        if (carry) w.push_back((u64)carry);
    }
    int cmp(const Big& o) const {
        size_t n = std::max(w.size(), o.w.size());
        for (size_t i = n; i-- > 0;) {
            u64 a = i < w.size() ? w[i] : 0, b = i < o.w.size() ? o.w[i] : 0;
            if (a != b) return a < b ? -1 : 1;
        }
        return 0;
    }
    Big sub(const Big& o) const {  // *this - o, requires *this >= o
        Big r;
        r.w.resize(w.size());
        u64 borrow = 0;
        for (size_t i = 0; i < w.size(); i++) {
            u64 b = i < o.w.size() ? o.w[i] : 0;
            lc::u128 t = (lc::u128)w[i] - b - borrow;
            r.w[i] = (u64)t;
            borrow = (t >> 64) ? 1 : 0;
        }
        return r;
    }
    Big half() const {
        Big r;
        r.w.resize(w.size());
        for (size_t i = 0; i < w.size(); i++) {
            r.w[i] = w[i] >> 1;
            if (i + 1 < w.size()) r.w[i] |= w[i + 1] << 63;
        }
        return r;
    }
    double to_double() const {
        long double v = 0;
        for (size_t i = w.size(); i-- > 0;) v = v * 18446744073709551616.0L + (long double)w[i];
        return (double)v;
    }
};
}  // namespace

// ------------------------------------------------------------------------------------ C ABI
extern "C" {

int lc_gen_primes(uint32_t log_n, uint32_t bits, uint32_t skip, uint32_t count, uint64_t* out) {
    if (!out || bits < 20 || bits > 62 || log_n < 1 || log_n > 20) return LC_EINVAL;
    std::vector<u64> v;
    if (!lc::ntt_primes((int)log_n, (int)bits, (int)skip, (int)count, v)) return LC_EINVAL;
    std::copy(v.begin(), v.end(), out);
    return LC_OK;
}

int lc_ctx_create(const lc_params* prm, int device, void* stream, const lc_allocator* alloc, lc_ctx** out) {
    if (!prm || !out || !prm->q || !prm->p) return LC_EINVAL;
    if (prm->log_n < 12 || prm->log_n > 16 || prm->n_q < 2 || prm->n_q > 24 || prm->n_p < 1 || prm->n_p > LC_MAX_P ||
        prm->dnum < 1 || prm->dnum > prm->n_q)
        return LC_EINVAL;
    lc_ctx* c = new (std::nothrow) lc_ctx();
    if (!c) return LC_ENOMEM;
    c->device = device;
    c->stream = static_cast<cudaStream_t>(stream);
    if (alloc && alloc->alloc && alloc->free) {
        c->alloc = *alloc;
        c->has_alloc = true;
    }
    c->log_n = (int)prm->log_n;
    c->N = (size_t)1 << prm->log_n;
    c->nq = (int)prm->n_q;
    c->np = (int)prm->n_p;
    c->dnum = (int)prm->dnum;
    c->debug = getenv("LC_DEBUG") != nullptr;
    c->alpha = (c->nq + c->dnum - 1) / c->dnum;
    if (c->alpha > LC_MAX_SRC || c->nq + c->np > LC_MAX_DST) {
        delete c;
        return LC_EINVAL;
    }
    const u64 twoN = 2 * (u64)c->N;
    for (uint32_t i = 0; i < prm->n_q; i++) c->mod.push_back(prm->q[i]);
    for (uint32_t i = 0; i < prm->n_p; i++) c->mod.push_back(prm->p[i]);
    for (u64 m : c->mod) {
        if (m >= ((u64)1 << 62) || m % twoN != 1 || !lc::probable_prime(m)) {
            delete c;
            return LC_EINVAL;
        }
    }
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return LC_ECUDA;
    }
    c->dev_err = static_cast<unsigned*>(lc_dev_alloc(c, 256));
    if (!c->dev_err || cudaMemset(c->dev_err, 0, 4) != cudaSuccess) {
        cudaGetLastError();
        lc_ctx_destroy(c);
        return LC_ENOMEM;
    }
    int st = build_tables(c);
    if (st != LC_OK) {
        lc_ctx_destroy(c);
        return st;
    }
    *out = c;
    return LC_OK;
}

void lc_ctx_destroy(lc_ctx* c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    lc_dev_free(c, c->tw_fwd);
    lc_dev_free(c, c->tw_inv);
    lc_dev_free(c, c->dev_err);
    lc_dev_free(c, c->mc);
    lc_dev_free(c, c->modup);
    lc_dev_free(c, c->moddown);
    lc_dev_free(c, c->rescale);
    lc_dev_free(c, c->scratch);
    lc_dev_free(c, c->stage);
    lc_dev_free(c, c->gather);
    lc_dev_free(c, c->enc_pos);
    lc_dev_free(c, c->enc_w256);
    lc_dev_free(c, c->enc_wbig);
    lc_dev_free(c, c->enc_buf);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    for (int d = 0; d < 2; d++)
        if (c->copy_stream[d]) {
            cudaStreamSynchronize(c->copy_stream[d]);
            cudaStreamDestroy(c->copy_stream[d]);
        }
    if (c->compute_mark) cudaEventDestroy(c->compute_mark);
    for (cudaEvent_t e : c->copy_events) cudaEventDestroy(e);
    delete c;
}

int lc_set_stream(lc_ctx* c, void* stream) {
    if (!c) return LC_EINVAL;
    c->stream = static_cast<cudaStream_t>(stream);
    return LC_OK;
}

int lc_sync(lc_ctx* c) {
    if (!c) return LC_EINVAL;
    LC_CUDA(c, cudaStreamSynchronize(c->stream));
    unsigned err = 0;
    LC_CUDA(c, cudaMemcpy(&err, c->dev_err, 4, cudaMemcpyDeviceToHost));
    if (err) {
        LC_CUDA(c, cudaMemset(c->dev_err, 0, 4));
        if (err & LC_ERR_TIMEOUT)
            return fail(c, LC_ETIMEOUT, "a bounded wait on the device gave up (code " + std::to_string(err) + ")");
        return fail(c, LC_EINVAL, "a wire-form residue was not below its prime (lc_unpack)");
    }
    return check_launch(c, "deferred");
}

const char* lc_last_error(const lc_ctx* c) { return c ? c->err.c_str() : "null context"; }

int lc_counters(lc_ctx* c, uint64_t* out, int reset) {
    if (!c || !out) return LC_EINVAL;
    out[0] = c->n_keyswitch;
    out[1] = c->n_modup;
    if (reset) c->n_keyswitch = c->n_modup = 0;
    return LC_OK;
}

int lc_pk_gen(lc_ctx* c, const int8_t* s, const uint64_t* a, const int32_t* e, uint64_t* pk) {
    clear_prior_error();
    if (!c || !s || !a || !e || !pk) return fail(c, LC_EINVAL, "lc_pk_gen: null argument");
    const size_t N = c->N;
    const int nq = c->nq;
    u64* t = lc_scratch(c, (size_t)N * 8 * (3 * nq + 2) + N * 8);
    if (!t) return fail(c, LC_ENOMEM, "scratch");
    u64* sr = t;
    u64* er = sr + (size_t)nq * N;
    u64* raw = er + (size_t)nq * N;  // int8/int32 staging
    std::vector<int> mods(nq);
    for (int i = 0; i < nq; i++) mods[i] = i;
    LC_CUDA(c, cudaMemcpyAsync(raw, s, N, cudaMemcpyHostToDevice, c->stream));
    op_to_rns_i8(c, reinterpret_cast<const int8_t*>(raw), 1, mods.data(), nq, sr);
    LC_CUDA(c, cudaStreamSynchronize(c->stream));
    LC_CUDA(c, cudaMemcpyAsync(raw, e, N * 4, cudaMemcpyHostToDevice, c->stream));
    op_to_rns_i32(c, reinterpret_cast<const int32_t*>(raw), 1, mods.data(), nq, er);
    u64* ap = pk + (size_t)nq * N;
    LC_CUDA(c, cudaMemcpyAsync(ap, a, (size_t)nq * N * 8, cudaMemcpyHostToDevice, c->stream));
    ntt_polys(c, sr, 1, nq, true);
    ntt_polys(c, er, 1, nq, true);
    ntt_polys(c, ap, 1, nq, true);
    op_key_combine(c, ap, sr, er, nullptr, nullptr, mods.data(), nq, pk);
    LC_CUDA(c, cudaStreamSynchronize(c->stream));
    return check_launch(c, "lc_pk_gen");
}

int lc_evk_create(lc_ctx* c, lc_evk** out) {
    if (!c || !out) return LC_EINVAL;
    lc_evk* k = new (std::nothrow) lc_evk();
    if (!k) return LC_ENOMEM;
    k->ctx = c;
    *out = k;
    return LC_OK;
}

void lc_evk_free(lc_evk* k) {
    if (!k) return;
    cudaStreamSynchronize(k->ctx->stream);
    for (auto& kv : k->keys) {
        lc_dev_free(k->ctx, kv.second.data);
        lc_dev_free(k->ctx, kv.second.qp);
    }
    delete k;
}

int lc_evk_add(lc_ctx* c, lc_evk* evk, const int8_t* s, int32_t rotation, const uint64_t* a, const int32_t* e) {
    clear_prior_error();
    if (!c || !evk || !s || !a || !e) return fail(c, LC_EINVAL, "lc_evk_add: null argument");
    const int32_t id = rotation < 0 ? -1 : rotation;
    if (rotation == 0) return fail(c, LC_EINVAL, "rotation 0 has no key");
    if (evk->keys.count(id)) return fail(c, LC_EBUSY, "key exists");
    const size_t N = c->N;
    const int rows = c->nq + c->np;
    const size_t keywords = (size_t)c->dnum * 2 * rows * N;
    u64* key = static_cast<u64*>(lc_dev_alloc(c, keywords * 8));
    if (!key) return fail(c, LC_ENOMEM, "key allocation");
    u64* t = lc_scratch(c, ((size_t)rows * 4 + 1) * N * 8 + keywords * 8);
    if (!t) {
        lc_dev_free(c, key);
        return fail(c, LC_ENOMEM, "scratch");
    }
    u64* sr = t;
    u64* st = sr + (size_t)rows * N;
    u64* er = st + (size_t)rows * N;
    u64* raw = er + (size_t)rows * N;
    u64* tmpkey = raw + N;
    std::vector<int> mods(rows);
    for (int i = 0; i < rows; i++) mods[i] = i;
    const uint64_t g = id < 0 ? 0 : galois_of(c, id);
    LC_CUDA(c, cudaMemcpyAsync(raw, s, N, cudaMemcpyHostToDevice, c->stream));
    op_to_rns_i8(c, reinterpret_cast<const int8_t*>(raw), 1, mods.data(), rows, sr);
    {
        RowMap m = rows_seq(rows);
        ntt_fwd_p(c, sr, 0, 1, m);
    }
    if (id < 0) op_square_rows(c, sr, st, mods.data(), rows);
    else op_permute_rows(c, sr, st, rows, g);
    std::vector<u64> Pmod(rows);
    u64* dst = id < 0 ? key : tmpkey;
    for (int j = 0; j < c->dnum; j++) {
        for (int r = 0; r < rows; r++) {
            const u64 m = c->mod[r];
            u64 P = 1 % m;
            for (int k = 0; k < c->np; k++) P = hmul(P, c->mod[c->nq + k] % m, m);
            const bool in_digit = r < c->nq && r / c->alpha == j;
            Pmod[r] = in_digit ? P : 0;
        }
        u64* kb = dst + (size_t)j * 2 * rows * N;
        u64* ka = kb + (size_t)rows * N;
        LC_CUDA(c, cudaStreamSynchronize(c->stream));
        LC_CUDA(c, cudaMemcpyAsync(ka, a + (size_t)j * rows * N, (size_t)rows * N * 8, cudaMemcpyHostToDevice, c->stream));
        LC_CUDA(c, cudaMemcpyAsync(raw, e + (size_t)j * N, N * 4, cudaMemcpyHostToDevice, c->stream));
        op_to_rns_i32(c, reinterpret_cast<const int32_t*>(raw), 1, mods.data(), rows, er);
        RowMap m = rows_seq(rows);
        ntt_fwd_p(c, ka, 0, 1, m);
        ntt_fwd_p(c, er, 0, 1, m);
        op_key_combine(c, ka, sr, er, st, Pmod.data(), mods.data(), rows, kb);
    }
    u64* qpkey = nullptr;
    if (id >= 0) {
        // store phi_g^-1(key): a hoisted rotation then permutes only its two output polys
        const uint64_t ginv = hpow(g, (u64)c->N / 2 - 1, 2 * (u64)c->N);  // g^(N/2-1) = g^-1 mod 2N
        op_permute_rows(c, tmpkey, key, c->dnum * 2 * rows, ginv);
        // and the un-permuted key, packed, for the one-ModDown group kernel
        qpkey = static_cast<u64*>(lc_dev_alloc(c, keywords * 8));
        if (!qpkey) {
            lc_dev_free(c, key);
            return fail(c, LC_ENOMEM, "key allocation");
        }
        op_pack_key(c, tmpkey, qpkey, keywords);
    }
    LC_CUDA(c, cudaStreamSynchronize(c->stream));
    int st_ = check_launch(c, "lc_evk_add");
    if (st_ != LC_OK) {
        lc_dev_free(c, key);
        lc_dev_free(c, qpkey);
        return st_;
    }
    evk->keys[id] = SwKey{key, g, qpkey};
    return LC_OK;
}

int lc_evk_import(lc_ctx* c, lc_evk* evk, int32_t rotation, const uint64_t* in) {
    clear_prior_error();
    if (!c || !evk || !in) return fail(c, LC_EINVAL, "lc_evk_import: null argument");
    const int32_t id = rotation < 0 ? -1 : rotation;
    if (rotation == 0) return fail(c, LC_EINVAL, "rotation 0 has no key");
    if (evk->keys.count(id)) return fail(c, LC_EBUSY, "key exists");
    const size_t N = c->N;
    const int rows = c->nq + c->np;
    const size_t keywords = (size_t)c->dnum * 2 * rows * N;
    // canonical residues only (row t of every digit and polynomial below its prime)
    for (size_t blk = 0; blk < (size_t)c->dnum * 2 * rows; blk++) {
        const u64 m = c->mod[blk % rows];
        const uint64_t* row = in + blk * N;
        for (size_t x = 0; x < N; x++)
            if (row[x] >= m) return fail(c, LC_EINVAL, "lc_evk_import: residue not below its prime");
    }
    u64* key = static_cast<u64*>(lc_dev_alloc(c, keywords * 8));
    if (!key) return fail(c, LC_ENOMEM, "key allocation");
    u64* qpkey = nullptr;
    u64* t = lc_scratch(c, keywords * 8);
    if (!t) {
        lc_dev_free(c, key);
        return fail(c, LC_ENOMEM, "scratch");
    }
    const uint64_t g = id < 0 ? 0 : galois_of(c, id);
    u64* dst = id < 0 ? key : t;
    LC_CUDA(c, cudaMemcpyAsync(dst, in, keywords * 8, cudaMemcpyHostToDevice, c->stream));
    ntt_fwd_p(c, dst, (size_t)rows * N, c->dnum * 2, rows_seq(rows));
    if (id >= 0) {  // the two device layouts of a rotation key, as lc_evk_add stores them
        const uint64_t ginv = hpow(g, (u64)c->N / 2 - 1, 2 * (u64)c->N);
        op_permute_rows(c, t, key, c->dnum * 2 * rows, ginv);
        qpkey = static_cast<u64*>(lc_dev_alloc(c, keywords * 8));
        if (!qpkey) {
            lc_dev_free(c, key);
            return fail(c, LC_ENOMEM, "key allocation");
        }
        op_pack_key(c, t, qpkey, keywords);
    }
    LC_CUDA(c, cudaStreamSynchronize(c->stream));
    const int st = check_launch(c, "lc_evk_import");
    if (st != LC_OK) {
        lc_dev_free(c, key);
        lc_dev_free(c, qpkey);
        return st;
    }
    evk->keys[id] = SwKey{key, g, qpkey};
    return LC_OK;
}

int lc_evk_export(lc_ctx* c, const lc_evk* evk, int32_t rotation, uint64_t* out) {
    clear_prior_error();
    if (!c || !evk || !out) return fail(c, LC_EINVAL, "lc_evk_export: null argument");
    const SwKey* k = find_key(evk, rotation < 0 ? -1 : rotation);
    if (!k) return fail(c, LC_EKEY, "key missing");
    const size_t N = c->N;
    const int rows = c->nq + c->np;
    const size_t words = (size_t)c->dnum * 2 * rows * N;
    u64* t = lc_scratch(c, words * 8);
    if (!t) return fail(c, LC_ENOMEM, "scratch");
    if (k->galois) op_permute_rows(c, k->data, t, c->dnum * 2 * rows, k->galois);
    else LC_CUDA(c, cudaMemcpyAsync(t, k->data, words * 8, cudaMemcpyDeviceToDevice, c->stream));
    RowMap m = rows_seq(rows);
    ntt_inv_p(c, t, (size_t)rows * N, c->dnum * 2, m);
    LC_CUDA(c, cudaMemcpyAsync(out, t, words * 8, cudaMemcpyDeviceToHost, c->stream));
    LC_CUDA(c, cudaStreamSynchronize(c->stream));
    return check_launch(c, "lc_evk_export");
}

int lc_encode(lc_ctx* c, const double* z, size_t len, double scale, int64_t* m_out) {
    if (!c || !m_out || (len && !z) || len > c->N / 2) return fail(c, LC_EINVAL, "lc_encode: bad argument");
    const size_t N = c->N, twoN = 2 * N;
    std::vector<std::complex<double>> A(twoN);
    u64 e = 1;
    for (size_t j = 0; j < N / 2; j++) {
        A[e] = std::complex<double>(j < len ? scale * z[j] : 0.0, 0.0);
        e = (e * 5) % twoN;
    }
    fft_inplace(A, false);
    for (size_t k = 0; k < N; k++) m_out[k] = (int64_t)std::nearbyint(2.0 / (double)N * A[k].real());
    return LC_OK;
}

int lc_decode(lc_ctx* c, const double* m, double scale, double* z_out) {
    if (!c || !m || !z_out) return fail(c, LC_EINVAL, "lc_decode: null argument");
    const size_t N = c->N, twoN = 2 * N;
    std::vector<std::complex<double>> A(twoN);
    for (size_t k = 0; k < N; k++) A[k] = m[k];
    fft_inplace(A, true);
    u64 e = 1;
    for (size_t j = 0; j < N / 2; j++) {
        z_out[j] = A[e].real() / scale;
        e = (e * 5) % twoN;
    }
    return LC_OK;
}

int lc_encrypt(lc_ctx* c, const uint64_t* pk, const int64_t* m, const int8_t* r, const int32_t* e0, const int32_t* e1,
               uint32_t count, uint64_t* out) {
    clear_prior_error();
    if (!c || !pk || !m || !r || !e0 || !e1 || !out) return fail(c, LC_EINVAL, "lc_encrypt: null argument");
    if (count == 0) return LC_OK;
    const size_t N = c->N;
    const int nq = c->nq;
    const size_t P = (size_t)nq * N;
    // process in slices that fit a modest scratch
    const uint32_t slice = std::max<uint32_t>(1, std::min<uint32_t>(count, 64));
    u64* t = lc_scratch(c, ((size_t)4 * slice * P + (size_t)slice * N) * 8);
    if (!t) return fail(c, LC_ENOMEM, "scratch");
    std::vector<int> mods(nq);
    for (int i = 0; i < nq; i++) mods[i] = i;
    for (uint32_t b0 = 0; b0 < count; b0 += slice) {
        const int B = (int)std::min(slice, count - b0);
        u64* mr = t;
        u64* rr = mr + (size_t)slice * P;
        u64* x0 = rr + (size_t)slice * P;
        u64* x1 = x0 + (size_t)slice * P;
        u64* raw = x1 + (size_t)slice * P;
        LC_CUDA(c, cudaStreamSynchronize(c->stream));
        LC_CUDA(c, cudaMemcpyAsync(raw, m + (size_t)b0 * N, (size_t)B * N * 8, cudaMemcpyHostToDevice, c->stream));
        op_to_rns_i64(c, reinterpret_cast<const int64_t*>(raw), B, mods.data(), nq, mr);
        LC_CUDA(c, cudaStreamSynchronize(c->stream));
        LC_CUDA(c, cudaMemcpyAsync(raw, r + (size_t)b0 * N, (size_t)B * N, cudaMemcpyHostToDevice, c->stream));
        op_to_rns_i8(c, reinterpret_cast<const int8_t*>(raw), B, mods.data(), nq, rr);
        LC_CUDA(c, cudaStreamSynchronize(c->stream));
        LC_CUDA(c, cudaMemcpyAsync(raw, e0 + (size_t)b0 * N, (size_t)B * N * 4, cudaMemcpyHostToDevice, c->stream));
        op_to_rns_i32(c, reinterpret_cast<const int32_t*>(raw), B, mods.data(), nq, x0);
        LC_CUDA(c, cudaStreamSynchronize(c->stream));
        LC_CUDA(c, cudaMemcpyAsync(raw, e1 + (size_t)b0 * N, (size_t)B * N * 4, cudaMemcpyHostToDevice, c->stream));
        op_to_rns_i32(c, reinterpret_cast<const int32_t*>(raw), B, mods.data(), nq, x1);
        if (B == (int)slice) {
            ntt_polys(c, mr, 4 * B, nq, true);  // mr, rr, x0, x1 are consecutive regions of `slice` polys
        } else {
            ntt_polys(c, mr, B, nq, true);
            ntt_polys(c, rr, B, nq, true);
            ntt_polys(c, x0, B, nq, true);
            ntt_polys(c, x1, B, nq, true);
        }
        op_enc_combine(c, mr, rr, x0, x1, pk, B, nq, out + (size_t)b0 * 2 * P);
    }
    LC_CUDA(c, cudaStreamSynchronize(c->stream));
    return check_launch(c, "lc_encrypt");
}

// encoder tables (first use) and a work buffer of at least `bytes`
static int encoder_ready(lc_ctx* c, size_t bytes) {
    const size_t N = c->N, M = 2 * N;
    if (!c->enc_pos) {
        std::vector<unsigned> pos(N / 2);
        u64 e = 1;
        for (size_t j = 0; j < N / 2; j++) {
            pos[j] = (unsigned)e;
            e = (e * 5) % M;
        }
        std::vector<double2> w256(256), wbig(M);
        for (int k = 0; k < 256; k++) w256[k] = make_double2(std::cos(2 * M_PI * k / 256), -std::sin(2 * M_PI * k / 256));
        for (size_t t = 0; t < M; t++)
            wbig[t] = make_double2(std::cos(2 * M_PI * (double)t / M), -std::sin(2 * M_PI * (double)t / M));
        c->enc_pos = static_cast<unsigned*>(lc_dev_alloc(c, pos.size() * 4));
        c->enc_w256 = static_cast<double2*>(lc_dev_alloc(c, 256 * sizeof(double2)));
        c->enc_wbig = static_cast<double2*>(lc_dev_alloc(c, M * sizeof(double2)));
        if (!c->enc_pos || !c->enc_w256 || !c->enc_wbig) return fail(c, LC_ENOMEM, "encoder tables");
        LC_CUDA(c, cudaMemcpy(c->enc_pos, pos.data(), pos.size() * 4, cudaMemcpyHostToDevice));
        LC_CUDA(c, cudaMemcpy(c->enc_w256, w256.data(), 256 * sizeof(double2), cudaMemcpyHostToDevice));
        LC_CUDA(c, cudaMemcpy(c->enc_wbig, wbig.data(), M * sizeof(double2), cudaMemcpyHostToDevice));
    }
    if (c->enc_buf_bytes < bytes) {
        if (c->capturing) return fail(c, LC_ENOMEM, "encoder buffer must be sized before a graph capture");
        LC_CUDA(c, cudaStreamSynchronize(c->stream));
        lc_dev_free(c, c->enc_buf);
        c->enc_buf = lc_dev_alloc(c, bytes);
        c->enc_buf_bytes = c->enc_buf ? bytes : 0;
        if (!c->enc_buf) return fail(c, LC_ENOMEM, "encoder buffer");
    }
    return LC_OK;
}

static const uint32_t kEncSlice = 64;

int lc_encode_dev(lc_ctx* c, const double* z_dev, uint32_t count, double scale, int64_t* m_dev) {
    clear_prior_error();
    if (!c || (count && (!z_dev || !m_dev))) return fail(c, LC_EINVAL, "lc_encode_dev: null argument");
    if (c->log_n != 15) return fail(c, LC_EINVAL, "lc_encode_dev: implemented for N = 2^15");
    if (count == 0) return LC_OK;
    const size_t N = c->N;
    const uint32_t slice = std::min(count, kEncSlice);
    if (int st = encoder_ready(c, (size_t)slice * 2 * N * sizeof(double2))) return st;
    for (uint32_t b0 = 0; b0 < count; b0 += slice) {
        const int B = (int)std::min(slice, count - b0);
        op_encode(c, z_dev + (size_t)b0 * (N / 2), B, scale, c->enc_pos, c->enc_w256, c->enc_wbig,
                  static_cast<double2*>(c->enc_buf), m_dev + (size_t)b0 * N);
    }
    return check_launch(c, "lc_encode_dev");
}

int lc_sample_enc(lc_ctx* c, uint64_t seed, uint64_t first, uint32_t count, int8_t* r, int32_t* e0, int32_t* e1) {
    clear_prior_error();
    if (!c || (count && (!r || !e0 || !e1))) return fail(c, LC_EINVAL, "lc_sample_enc: null argument");
    if (count == 0) return LC_OK;
    const size_t n = (size_t)count * c->N;
    unsigned char* t = reinterpret_cast<unsigned char*>(lc_scratch(c, n * 9 + 64));
    if (!t) return fail(c, LC_ENOMEM, "scratch");
    int32_t* d0 = reinterpret_cast<int32_t*>(t);
    int32_t* d1 = d0 + n;
    int8_t* dr = reinterpret_cast<int8_t*>(d1 + n);
    op_sample_enc(c, seed, first, (int)count, dr, d0, d1);
    LC_CUDA(c, cudaMemcpyAsync(r, dr, n, cudaMemcpyDeviceToHost, c->stream));
    LC_CUDA(c, cudaMemcpyAsync(e0, d0, n * 4, cudaMemcpyDeviceToHost, c->stream));
    LC_CUDA(c, cudaMemcpyAsync(e1, d1, n * 4, cudaMemcpyDeviceToHost, c->stream));
    LC_CUDA(c, cudaStreamSynchronize(c->stream));
    return check_launch(c, "lc_sample_enc");
}

// encryption of `count` device plaintexts (m_dev, [count][N] int64) or constant-slot values
// (w_dev, [count] doubles, coefficient 0 = round(w scale)) with device randomness; no host
// synchronisation, so it may be captured in a graph (scratch must be sized beforehand).
static int encrypt_seeded(lc_ctx* c, const uint64_t* pk, const int64_t* m_dev, const double* w_dev, double scale,
                          uint32_t count, uint64_t seed, uint64_t first, uint64_t* out) {
    const size_t N = c->N;
    const int nq = c->nq;
    const size_t P = (size_t)nq * N;
    const uint32_t slice = std::max<uint32_t>(1, std::min<uint32_t>(count, 64));
    // 4 RNS regions + int64 plaintexts (N words) + two int32 error rows (N words) + ternary bytes
    const size_t words = (size_t)4 * slice * P + (size_t)slice * N * 3 + 64;
    u64* t = lc_scratch(c, words * 8);
    if (!t) return fail(c, LC_ENOMEM, "scratch");
    std::vector<int> mods(nq);
    for (int i = 0; i < nq; i++) mods[i] = i;
    for (uint32_t b0 = 0; b0 < count; b0 += slice) {
        const int B = (int)std::min(slice, count - b0);
        u64* mr = t;
        u64* rr = mr + (size_t)slice * P;
        u64* x0 = rr + (size_t)slice * P;
        u64* x1 = x0 + (size_t)slice * P;
        int64_t* mplain = reinterpret_cast<int64_t*>(x1 + (size_t)slice * P);  // [slice][N]
        int32_t* de0 = reinterpret_cast<int32_t*>(mplain + (size_t)slice * N);
        int32_t* de1 = de0 + (size_t)slice * N;
        int8_t* dr = reinterpret_cast<int8_t*>(de1 + (size_t)slice * N);
        const int64_t* mb = m_dev ? m_dev + (size_t)b0 * N : mplain;
        if (!m_dev) op_const_plain(c, w_dev + b0, B, scale, mplain);
        op_to_rns_i64(c, mb, B, mods.data(), nq, mr);
        op_sample_enc(c, seed, first + b0, B, dr, de0, de1);
        op_to_rns_i8(c, dr, B, mods.data(), nq, rr);
        op_to_rns_i32(c, de0, B, mods.data(), nq, x0);
        op_to_rns_i32(c, de1, B, mods.data(), nq, x1);
        if (B == (int)slice) {
            ntt_polys(c, mr, 4 * B, nq, true);
        } else {
            ntt_polys(c, mr, B, nq, true);
            ntt_polys(c, rr, B, nq, true);
            ntt_polys(c, x0, B, nq, true);
            ntt_polys(c, x1, B, nq, true);
        }
        op_enc_combine(c, mr, rr, x0, x1, pk, B, nq, out + (size_t)b0 * 2 * P);
    }
    return check_launch(c, "encrypt (device randomness)");
}

int lc_encrypt_seeded(lc_ctx* c, const uint64_t* pk, const int64_t* m_dev, uint32_t count, uint64_t seed,
                      uint64_t first, uint64_t* out) {
    clear_prior_error();
    if (!c || !pk || !out || (count && !m_dev)) return fail(c, LC_EINVAL, "lc_encrypt_seeded: null argument");
    if (count == 0) return LC_OK;
    return encrypt_seeded(c, pk, m_dev, nullptr, 0.0, count, seed, first, out);
}

int lc_encrypt_const_seeded(lc_ctx* c, const uint64_t* pk, const double* w_dev, uint32_t count, double scale,
                            uint64_t seed, uint64_t first, uint64_t* out) {
    clear_prior_error();
    if (!c || !pk || !out || (count && !w_dev)) return fail(c, LC_EINVAL, "lc_encrypt_const_seeded: null argument");
    if (count == 0) return LC_OK;
    return encrypt_seeded(c, pk, nullptr, w_dev, scale, count, seed, first, out);
}

int lc_encode_encrypt_seeded(lc_ctx* c, const uint64_t* pk, const double* z_dev, uint32_t count, double scale,
                             uint64_t seed, uint64_t first, uint64_t* out) {
    clear_prior_error();
    if (!c || !pk || !out || (count && !z_dev)) return fail(c, LC_EINVAL, "lc_encode_encrypt_seeded: null argument");
    if (c->log_n != 15) return fail(c, LC_EINVAL, "lc_encode_encrypt_seeded: implemented for N = 2^15");
    if (count == 0) return LC_OK;
    const size_t N = c->N, P = (size_t)c->nq * N;
    const uint32_t slice = std::min(count, kEncSlice);
    // work buffer: the FFT array, then the integer plaintexts of one slice
    const size_t fft_bytes = (size_t)slice * 2 * N * sizeof(double2);
    if (int st = encoder_ready(c, fft_bytes + (size_t)slice * N * 8)) return st;
    int64_t* m = reinterpret_cast<int64_t*>(static_cast<char*>(c->enc_buf) + fft_bytes);
    for (uint32_t b0 = 0; b0 < count; b0 += slice) {
        const uint32_t B = std::min(slice, count - b0);
        op_encode(c, z_dev + (size_t)b0 * (N / 2), (int)B, scale, c->enc_pos, c->enc_w256, c->enc_wbig,
                  static_cast<double2*>(c->enc_buf), m);
        if (int st = encrypt_seeded(c, pk, m, nullptr, 0.0, B, seed, first + b0, out + (size_t)b0 * 2 * P)) return st;
    }
    return check_launch(c, "lc_encode_encrypt_seeded");
}

int lc_decrypt(lc_ctx* c, const int8_t* s, const uint64_t* ct, uint32_t deg, uint32_t level, uint64_t* res_out) {
    clear_prior_error();
    if (!c || !s || !ct || !res_out || deg < 2 || deg > 3) return fail(c, LC_EINVAL, "lc_decrypt: bad argument");
    if ((int)level >= c->nq) return fail(c, LC_ELEVEL, "level out of range");
    const size_t N = c->N;
    const int nl = (int)level + 1;
    u64* t = lc_scratch(c, ((size_t)2 * nl + 1) * N * 8);
    if (!t) return fail(c, LC_ENOMEM, "scratch");
    u64* sr = t;
    u64* acc = sr + (size_t)nl * N;
    u64* raw = acc + (size_t)nl * N;
    std::vector<int> mods(nl);
    for (int i = 0; i < nl; i++) mods[i] = i;
    LC_CUDA(c, cudaMemcpyAsync(raw, s, N, cudaMemcpyHostToDevice, c->stream));
    op_to_rns_i8(c, reinterpret_cast<const int8_t*>(raw), 1, mods.data(), nl, sr);
    ntt_polys(c, sr, 1, nl, true);
    op_dec_combine(c, ct, sr, (int)deg, nl, acc);
    ntt_polys(c, acc, 1, nl, false);
    LC_CUDA(c, cudaMemcpyAsync(res_out, acc, (size_t)nl * N * 8, cudaMemcpyDeviceToHost, c->stream));
    LC_CUDA(c, cudaStreamSynchronize(c->stream));
    return check_launch(c, "lc_decrypt");
}

int lc_decrypt_const(lc_ctx* c, const int8_t* s, const uint64_t* cts, uint32_t count, uint32_t level, double scale,
                     double* out) {
    if (!c || !s || !cts || !out || (int)level >= c->nq) return fail(c, LC_EINVAL, "lc_decrypt_const: bad argument");
    if (count == 0) return LC_OK;
    clear_prior_error();
    const size_t N = c->N;
    u64* t = lc_scratch(c, (2 * N + count + 8) * 8);
    if (!t) return fail(c, LC_ENOMEM, "scratch");
    u64* s0 = t;
    u64* raw = s0 + N;
    u64* res = raw + N;
    const int mods[1] = {0};
    LC_CUDA(c, cudaMemcpyAsync(raw, s, N, cudaMemcpyHostToDevice, c->stream));
    op_to_rns_i8(c, reinterpret_cast<const int8_t*>(raw), 1, mods, 1, s0);
    RowMap m = rows_seq(1);
    ntt_fwd_p(c, s0, N, 1, m);
    op_const_coef0(c, cts, (size_t)2 * (level + 1) * N, (int)count, s0, res);
    std::vector<u64> h(count);
    LC_CUDA(c, cudaMemcpyAsync(h.data(), res, count * 8, cudaMemcpyDeviceToHost, c->stream));
    LC_CUDA(c, cudaStreamSynchronize(c->stream));
    const u64 q0 = c->mod[0];
    for (uint32_t k = 0; k < count; k++) {
        const double v = h[k] > q0 / 2 ? -(double)(q0 - h[k]) : (double)h[k];
        out[k] = v / scale;
    }
    return check_launch(c, "lc_decrypt_const");
}

// ------------------------------------------------------------------------------- KGC on the device
struct lc_kgc {
    lc_ctx* c = nullptr;
    u64* s0 = nullptr;  // secret mod q0, evaluation domain (limb 0)
};

int lc_kgc_create(lc_ctx* c, const int8_t* s, lc_kgc** out) {
    clear_prior_error();
    if (!c || !s || !out) return fail(c, LC_EINVAL, "lc_kgc_create: null argument");
    const size_t N = c->N;
    auto* k = new lc_kgc;
    k->c = c;
    k->s0 = static_cast<u64*>(lc_dev_alloc(c, N * 8));
    u64* raw = lc_scratch(c, N * 8);
    if (!k->s0 || !raw) {
        if (k->s0) lc_dev_free(c, k->s0);
        delete k;
        return fail(c, LC_ENOMEM, "lc_kgc_create");
    }
    const int mods[1] = {0};
    LC_CUDA(c, cudaMemcpyAsync(raw, s, N, cudaMemcpyHostToDevice, c->stream));
    op_to_rns_i8(c, reinterpret_cast<const int8_t*>(raw), 1, mods, 1, k->s0);
    RowMap m = rows_seq(1);
    ntt_fwd_p(c, k->s0, N, 1, m);
    LC_CUDA(c, cudaStreamSynchronize(c->stream));
    *out = k;
    return check_launch(c, "lc_kgc_create");
}

void lc_kgc_free(lc_kgc* k) {
    if (!k) return;
    cudaStreamSynchronize(k->c->stream);
    lc_dev_free(k->c, k->s0);
    delete k;
}

int lc_kgc_readout(lc_ctx* c, const lc_kgc* k, const uint64_t* cts, uint32_t count, uint32_t level, double scale,
                   double* out_dev) {
    if (!c || !k || !cts || !out_dev || (int)level >= c->nq) return fail(c, LC_EINVAL, "lc_kgc_readout: bad argument");
    if (count == 0) return LC_OK;
    u64* res = lc_scratch(c, ((size_t)count + 8) * 8);
    if (!res) return fail(c, LC_ENOMEM, "scratch");
    op_const_coef0(c, cts, (size_t)2 * (level + 1) * c->N, (int)count, k->s0, res);
    op_readout_finish(c, res, (int)count, scale, out_dev);
    return check_launch(c, "lc_kgc_readout");
}

int lc_kgc_krum(lc_ctx* c, const double* dist_dev, uint32_t n, uint32_t f, uint32_t n_select, int average,
                double* w_dev, int32_t* sel_dev) {
    if (!c || !dist_dev || !w_dev || !sel_dev || n < 1 || n > 256 || n_select < 1 || n_select > n)
        return fail(c, LC_EINVAL, "lc_kgc_krum: bad argument (1 <= n_select <= n <= 256)");
    op_krum(c, dist_dev, (int)n, (int)f, (int)n_select, average ? 1 : 0, w_dev, sel_dev);
    return check_launch(c, "lc_kgc_krum");
}

int lc_crt_to_double(lc_ctx* c, const uint64_t* res, uint32_t level, double* m_out) {
    if (!c || !res || !m_out || (int)level >= c->nq) return fail(c, LC_EINVAL, "lc_crt_to_double: bad argument");
    const size_t N = c->N;
    const int nl = (int)level + 1;
    // Garner mixed radix: x = v0 + v1 q0 + v2 q0 q1 + ...
    std::vector<std::vector<u64>> inv(nl, std::vector<u64>(nl, 0));
    for (int i = 0; i < nl; i++)
        for (int k = 0; k < i; k++) inv[k][i] = hinv(c->mod[k] % c->mod[i], c->mod[i]);
    Big Q;
    Q.w = {1};
    for (int i = 0; i < nl; i++) Q.mul_add(c->mod[i], 0);
    const Big half = Q.half();
    std::vector<u64> v(nl);
    for (size_t x = 0; x < N; x++) {
        for (int i = 0; i < nl; i++) {
            const u64 qi = c->mod[i];
            u64 t = res[(size_t)i * N + x] % qi;
            for (int k = 0; k < i; k++) {
                t = (t + qi - v[k] % qi) % qi;
                t = hmul(t, inv[k][i], qi);
            }
            v[i] = t;
        }
        Big X;
        X.w = {v[nl - 1]};
        for (int i = nl - 2; i >= 0; i--) X.mul_add(c->mod[i], v[i]);
        if (X.cmp(half) > 0) m_out[x] = -Q.sub(X).to_double();
        else m_out[x] = X.to_double();
    }
    return LC_OK;
}

int lc_to_coeff(lc_ctx* c, uint64_t* data, uint32_t n_polys, uint32_t level) {
    clear_prior_error();
    if (!c || !data || (int)level >= c->nq) return fail(c, LC_EINVAL, "lc_to_coeff: bad argument");
    ntt_polys(c, data, (int)n_polys, (int)level + 1, false);
    return check_launch(c, "lc_to_coeff");
}

int lc_to_eval(lc_ctx* c, uint64_t* data, uint32_t n_polys, uint32_t level) {
    clear_prior_error();
    if (!c || !data || (int)level >= c->nq) return fail(c, LC_EINVAL, "lc_to_eval: bad argument");
    ntt_polys(c, data, (int)n_polys, (int)level + 1, true);
    return check_launch(c, "lc_to_eval");
}

int lc_add(lc_ctx* c, const uint64_t* a, const uint64_t* b, uint32_t n_polys, uint32_t level, uint64_t* out) {
    clear_prior_error();
    if (!c || !a || !b || !out || (int)level >= c->nq) return fail(c, LC_EINVAL, "lc_add: bad argument");
    op_addsub(c, a, b, out, (int)n_polys, (int)level + 1, false);
    return check_launch(c, "lc_add");
}

int lc_sub(lc_ctx* c, const uint64_t* a, const uint64_t* b, uint32_t n_polys, uint32_t level, uint64_t* out) {
    clear_prior_error();
    if (!c || !a || !b || !out || (int)level >= c->nq) return fail(c, LC_EINVAL, "lc_sub: bad argument");
    op_addsub(c, a, b, out, (int)n_polys, (int)level + 1, true);
    return check_launch(c, "lc_sub");
}

int lc_tensor(lc_ctx* c, const uint64_t* a, const uint64_t* b, uint32_t level, uint64_t* out) {
    clear_prior_error();
    if (!c || !a || !b || !out || (int)level >= c->nq) return fail(c, LC_EINVAL, "lc_tensor: bad argument");
    op_tensor(c, a, b, out, (int)level + 1);
    return check_launch(c, "lc_tensor");
}

int lc_relin(lc_ctx* c, const lc_evk* evk, const uint64_t* ct3, uint32_t count, uint32_t level, uint64_t* out) {
    clear_prior_error();
    if (!c || !evk || !ct3 || !out || (int)level >= c->nq) return fail(c, LC_EINVAL, "lc_relin: bad argument");
    if (count == 0) return LC_OK;
    u64* t = lc_scratch(c, ks_words(c, (int)count, (int)level) * 8);
    if (!t) return fail(c, LC_ENOMEM, "scratch");
    int st = do_relin(c, evk, ct3, (int)count, (int)level, out, t);
    if (st) return st;
    return check_launch(c, "lc_relin");
}

int lc_rescale(lc_ctx* c, const uint64_t* ct, uint32_t count, uint32_t deg, uint32_t level, uint64_t* out) {
    clear_prior_error();
    if (!c || !ct || !out || level < 1 || (int)level >= c->nq || deg < 1 || deg > 3)
        return fail(c, LC_EINVAL, "lc_rescale: bad argument");
    if (count == 0) return LC_OK;
    u64* t = lc_scratch(c, rescale_words(c, (int)count, (int)deg, (int)level) * 8);
    if (!t) return fail(c, LC_ENOMEM, "scratch");
    do_rescale(c, ct, (int)count, (int)deg, (int)level, out, t);
    return check_launch(c, "lc_rescale");
}

int lc_rotate(lc_ctx* c, const lc_evk* evk, const uint64_t* ct, uint32_t level, uint32_t n_rot, const int32_t* rots,
              uint64_t* out) {
    clear_prior_error();
    if (!c || !evk || !ct || !out || (n_rot && !rots) || (int)level >= c->nq)
        return fail(c, LC_EINVAL, "lc_rotate: bad argument");
    if (n_rot == 0) return LC_OK;
    const size_t P = (size_t)(level + 1) * c->N;
    std::vector<const SwKey*> keys(n_rot);
    for (uint32_t r = 0; r < n_rot; r++) {
        keys[r] = rots[r] > 0 ? find_key(evk, rots[r]) : nullptr;
        if (!keys[r]) return fail(c, LC_EKEY, "rotation key missing");
    }
    const size_t kw = ks_words(c, 1, (int)level);
    u64* t = lc_scratch(c, (kw + 2 * P) * 8);
    if (!t) return fail(c, LC_ENOMEM, "scratch");
    KsBufs kb = ks_layout(c, t, 1, (int)level);
    u64* w = t + kw;
    ks_modup(c, ct + P, 2 * P, 1, (int)level, kb);
    for (uint32_t r = 0; r < n_rot; r++) {
        ks_apply(c, ct + P, 2 * P, 1, (int)level, keys[r]->data, kb, ct, nullptr, 2 * P, w, 2 * P);
        op_gather(c, w, out + (size_t)r * 2 * P, 2, (int)level + 1, keys[r]->galois, false);
    }
    return check_launch(c, "lc_rotate");
}

int lc_rotate_sum(lc_ctx* c, const lc_evk* evk, uint64_t* cts, uint32_t count, uint32_t level, uint32_t n_groups,
                  const uint32_t* groups, uint32_t flags) {
    clear_prior_error();
    if (!c || !evk || !cts || (int)level >= c->nq) return fail(c, LC_EINVAL, "lc_rotate_sum: bad argument");
    if (count == 0 || n_groups == 0) return LC_OK;
    int maxg = 1;
    for (uint32_t i = 0; i < n_groups; i++) maxg = std::max(maxg, (int)(groups ? groups[i] : 1));
    const bool qp = (flags & LC_HOIST_QP_SUM) != 0;
    if (maxg > (qp ? 4 : 8)) return fail(c, LC_EINVAL, "group too large (one-ModDown groups: at most 4 bits)");
    u64* t = lc_scratch(c, rotsum_words(c, (int)count, (int)level, maxg, qp) * 8);
    if (!t) return fail(c, LC_ENOMEM, "scratch");
    int st = do_rotate_sum(c, evk, cts, (int)count, (int)level, (int)n_groups, groups, t, qp);
    if (st) return st;
    return check_launch(c, "lc_rotate_sum");
}

int lc_memcpy_h2d(lc_ctx* c, uint64_t* dst, const void* src, size_t bytes) {
    if (!c || (!dst && bytes) || (!src && bytes)) return fail(c, LC_EINVAL, "lc_memcpy_h2d: null argument");
    LC_CUDA(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->stream));
    return LC_OK;
}

int lc_memcpy_d2h(lc_ctx* c, void* dst, const uint64_t* src, size_t bytes) {
    if (!c || (!dst && bytes) || (!src && bytes)) return fail(c, LC_EINVAL, "lc_memcpy_d2h: null argument");
    LC_CUDA(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, c->stream));
    return LC_OK;
}

int lc_copy_async(lc_ctx* c, void* dst, const void* src, size_t bytes, int dir, uint64_t* ticket) {
    if (!c || !ticket || (dir != LC_H2D && dir != LC_D2H) || (bytes && (!dst || !src)))
        return fail(c, LC_EINVAL, "lc_copy_async: bad argument");
    if (c->capturing) return fail(c, LC_EBUSY, "lc_copy_async: not inside a graph capture");
    if (!c->copy_stream[dir]) LC_CUDA(c, cudaStreamCreateWithFlags(&c->copy_stream[dir], cudaStreamNonBlocking));
    if (!c->compute_mark) LC_CUDA(c, cudaEventCreateWithFlags(&c->compute_mark, cudaEventDisableTiming));
    size_t slot;
    if (!c->copy_free.empty()) {
        slot = c->copy_free.back();
        c->copy_free.pop_back();
    } else {
        cudaEvent_t ev;
        LC_CUDA(c, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        c->copy_events.push_back(ev);
        c->copy_busy.push_back(0);
        slot = c->copy_events.size() - 1;
    }
    // ordered after everything enqueued on the context's stream so far
    LC_CUDA(c, cudaEventRecord(c->compute_mark, c->stream));
    LC_CUDA(c, cudaStreamWaitEvent(c->copy_stream[dir], c->compute_mark, 0));
    LC_CUDA(c, cudaMemcpyAsync(dst, src, bytes, dir == LC_H2D ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost,
                               c->copy_stream[dir]));
    LC_CUDA(c, cudaEventRecord(c->copy_events[slot], c->copy_stream[dir]));
    c->copy_busy[slot] = 1;
    *ticket = slot;
    return LC_OK;
}

int lc_copy_wait(lc_ctx* c, uint64_t ticket) {
    if (!c || ticket >= c->copy_events.size() || !c->copy_busy[ticket])
        return fail(c, LC_EINVAL, "lc_copy_wait: unknown or already waited ticket");
    LC_CUDA(c, cudaStreamWaitEvent(c->stream, c->copy_events[ticket], 0));
    // the wait binds to the record made by lc_copy_async, so the slot can be recorded again
    c->copy_busy[ticket] = 0;
    c->copy_free.push_back(ticket);
    return LC_OK;
}

int lc_launches(uint64_t* out) {
    if (!out) return LC_EINVAL;
    *out = g_lc_launches.load();
    return LC_OK;
}

int lc_profile(lc_ctx* c, int start, double* ms, double* bytes, uint64_t* launches) {
    if (!c) return LC_EINVAL;
    if (start) {
        c->prof.clear();
        c->ev_used = 0;
        c->prof_on = true;
        return LC_OK;
    }
    c->prof_on = false;
    LC_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int k = 0; k < PROF_N; k++) {
        if (ms) ms[k] = 0;
        if (bytes) bytes[k] = 0;
        if (launches) launches[k] = 0;
    }
    for (const ProfRec& r : c->prof) {
        float t = 0;
        cudaEventElapsedTime(&t, r.a, r.b);
        if (ms) ms[r.cls] += t;
        if (bytes) bytes[r.cls] += r.bytes;
        if (launches) launches[r.cls] += 1;
    }
    c->prof.clear();
    c->ev_used = 0;
    return check_launch(c, "lc_profile");
}

// ------------------------------------------------------------------------------------ the method
static int max_batch_for(lc_ctx* c, size_t words_per_item, size_t budget_words) {
    size_t b = budget_words / std::max<size_t>(1, words_per_item);
    b = std::max<size_t>(1, std::min<size_t>(b, 4096));
    if (c->max_batch) b = std::min<size_t>(b, c->max_batch);
    return (int)b;
}

struct lc_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t launches = 0;
};

int lc_graph_begin(lc_ctx* c) {
    if (!c) return LC_EINVAL;
    if (!c->stream) return fail(c, LC_EINVAL, "graph capture needs a context stream other than the legacy default");
    if (c->capturing) return fail(c, LC_EBUSY, "already capturing");
    LC_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    c->capturing = true;
    c->capture_launches0 = g_lc_launches.load();
    return LC_OK;
}

int lc_graph_end(lc_ctx* c, lc_graph** out) {
    if (!c || !out) return LC_EINVAL;
    if (!c->capturing) return fail(c, LC_EINVAL, "not capturing");
    c->capturing = false;
    lc_graph* g = new (std::nothrow) lc_graph();
    if (!g) return LC_ENOMEM;
    cudaError_t e = cudaStreamEndCapture(c->stream, &g->graph);
    if (e != cudaSuccess) {
        delete g;
        cudaGetLastError();
        return fail(c, LC_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
    }
    e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g->graph);
        delete g;
        cudaGetLastError();
        return fail(c, LC_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    }
    g->launches = g_lc_launches.load() - c->capture_launches0;
    *out = g;
    return LC_OK;
}

int lc_graph_launch(lc_ctx* c, const lc_graph* g) {
    if (!c || !g) return LC_EINVAL;
    LC_CUDA(c, cudaGraphLaunch(g->exec, c->stream));
    g_lc_launches += g->launches;
    return LC_OK;
}

void lc_graph_free(lc_graph* g) {
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
}

int lc_set_max_batch(lc_ctx* c, uint32_t max_items) {
    if (!c) return LC_EINVAL;
    c->max_batch = max_items;
    return LC_OK;
}

int lc_set_tuning(lc_ctx* c, uint32_t knob, int32_t value) {
    if (!c) return LC_EINVAL;
    bool ok = false;
    switch (knob) {
        case LC_TUNE_NTT_ROW_MINB: ok = value == 4 || value == 5 || value == 6; break;
        case LC_TUNE_NTT_COL_MINB: ok = value == 1 || value == 6 || value == 7 || value == 8; break;
        case LC_TUNE_GROUP_SPLIT_ITEMS:
        case LC_TUNE_GROUP_WIDE_ITEMS: ok = value == 1 || value == 2; break;
        case LC_TUNE_TENSOR_WARPS: ok = value == 8 || value == 12 || value == 16; break;
        case LC_TUNE_NTT_ROW_TMA:
        case LC_TUNE_GROUP_KARATSUBA: ok = value == 0 || value == 1; break;
        default: break;
    }
    if (!ok) return fail(c, LC_EINVAL, "lc_set_tuning: knob " + std::to_string(knob) + " has no option " +
                                           std::to_string(value));
    c->tune[knob] = value;
    return LC_OK;
}

int lc_get_tuning(const lc_ctx* c, uint32_t knob, int32_t* value) {
    if (!c || !value || knob < LC_TUNE_NTT_ROW_MINB || knob > LC_TUNE_GROUP_KARATSUBA) return LC_EINVAL;
    *value = c->tune[knob];
    return LC_OK;
}

int lc_alu_probe(lc_ctx* c, uint32_t kind, uint32_t iters, uint32_t blocks_per_sm, double* ms, double* ops) {
    clear_prior_error();
    if (!c || !ms || !ops || kind > LC_PROBE_NTT_BFLY || iters == 0 || blocks_per_sm < 1 || blocks_per_sm > 32)
        return fail(c, LC_EINVAL, "lc_alu_probe: bad argument");
    int sms = 0;
    LC_CUDA(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
    const int blocks = sms * (int)blocks_per_sm;
    cudaEvent_t e0, e1;
    LC_CUDA(c, cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(c, LC_ECUDA, "lc_alu_probe: event creation failed");
    }
    auto* sink = static_cast<unsigned long long*>(lc_dev_alloc(c, sizeof(unsigned long long)));
    if (!sink) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return fail(c, LC_ENOMEM, "lc_alu_probe: allocation failed");
    }
    auto launch = [&] {
        if (kind == LC_PROBE_IMAD) probe_imad(blocks, iters, sink, c->stream);
        else if (kind == LC_PROBE_IMAD_WIDE) probe_imad_wide(blocks, iters, sink, c->stream);
        else probe_ntt_bfly(blocks, iters, sink, c->stream);
    };
    launch();  // warm: module loaded, clocks up
    cudaEventRecord(e0, c->stream);
    launch();
    cudaEventRecord(e1, c->stream);
    g_lc_launches += 2;
    cudaError_t st = cudaEventSynchronize(e1);
    float t = 0.f;
    if (st == cudaSuccess) st = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    lc_dev_free(c, sink);
    LC_CUDA(c, st);
    *ms = t;
    *ops = (double)blocks * kProbeThreads * iters * (kind == LC_PROBE_NTT_BFLY ? 32.0 : 64.0);
    return check_launch(c, "lc_alu_probe");
}

static bool wire_map(lc_ctx* c, uint32_t deg, uint32_t level, WireMap& m) {
    if (deg < 1 || deg > 3 || (int)level >= c->nq || level + 1 > LC_WIRE_MAX_LIMBS || c->log_n < 4) return false;
    m = WireMap{};
    m.log_n = c->log_n;
    m.nl = (int)level + 1;
    size_t off = 0;
    for (int i = 0; i < m.nl; i++) {
        int bits = 0;
        for (u64 v = c->mod[i] - 1; v; v >>= 1) bits++;
        m.w[i] = std::min(8, std::max(4, (bits + 7) / 8));
        m.off[i] = off;
        m.q[i] = c->mod[i];
        off += (size_t)c->N * m.w[i];
    }
    m.poly_bytes = off;
    return true;
}

int lc_wire_bytes(lc_ctx* c, uint32_t deg, uint32_t level, uint64_t* bytes) {
    WireMap m;
    if (!c || !bytes || !wire_map(c, deg, level, m)) return fail(c, LC_EINVAL, "lc_wire_bytes: bad argument");
    *bytes = (uint64_t)m.poly_bytes * deg;
    return LC_OK;
}

int lc_pack(lc_ctx* c, const uint64_t* in, uint32_t count, uint32_t deg, uint32_t level, uint8_t* out) {
    clear_prior_error();
    WireMap m;
    if (!c || !in || !out || !wire_map(c, deg, level, m) || is_host_ptr(in) || is_host_ptr(out) ||
        (reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) % 16)
        return fail(c, LC_EINVAL, "lc_pack: bad argument (device buffers, 16-byte aligned)");
    wire_pack(in, out, (size_t)count * deg, m, c->stream);
    g_lc_launches += count ? 1 : 0;
    return check_launch(c, "lc_pack");
}

int lc_unpack(lc_ctx* c, const uint8_t* in, uint32_t count, uint32_t deg, uint32_t level, uint64_t* out) {
    clear_prior_error();
    WireMap m;
    if (!c || !in || !out || !wire_map(c, deg, level, m) || is_host_ptr(in) || is_host_ptr(out) ||
        (reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) % 16)
        return fail(c, LC_EINVAL, "lc_unpack: bad argument (device buffers, 16-byte aligned)");
    wire_unpack(in, out, (size_t)count * deg, m, c->dev_err, c->stream);
    g_lc_launches += count ? 1 : 0;
    return check_launch(c, "lc_unpack");
}

int lc_wait_selftest(lc_ctx* c, int never_arrive, uint32_t max_polls) {
    clear_prior_error();
    if (!c || max_polls == 0) return fail(c, LC_EINVAL, "lc_wait_selftest: bad argument");
    auto* buf = static_cast<unsigned long long*>(lc_dev_alloc(c, 128));
    if (!buf) return fail(c, LC_ENOMEM, "lc_wait_selftest: allocation failed");
    unsigned long long pattern[8], back[8] = {};
    for (int i = 0; i < 8; i++) pattern[i] = 0x9e3779b97f4a7c15ull * (unsigned long long)(i + 1);
    cudaError_t e = cudaMemcpyAsync(buf, pattern, sizeof(pattern), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(buf + 8, 0, 64, c->stream);
    if (e == cudaSuccess) {
        wait_selftest(buf, buf + 8, never_arrive, max_polls, c->dev_err, c->stream);
        g_lc_launches += 1;
        e = cudaMemcpyAsync(back, buf + 8, sizeof(back), cudaMemcpyDeviceToHost, c->stream);
    }
    const int st = e == cudaSuccess ? lc_sync(c) : fail(c, LC_ECUDA, cudaGetErrorString(e));
    lc_dev_free(c, buf);
    if (st) return st;
    if (std::memcmp(back, pattern, sizeof(back)) != 0)
        return fail(c, LC_ECUDA, "lc_wait_selftest: the bulk copy delivered wrong bytes");
    return LC_OK;
}

int lc_distances(lc_ctx* c, const lc_evk* evk, const uint64_t* cts, uint32_t n, uint32_t chunks, double scale,
                 uint32_t mode, uint32_t n_groups, const uint32_t* groups, uint64_t* out, double* out_scale) {
    clear_prior_error();
    if (!c || !evk || !cts || !out || n < 2 || chunks == 0) return fail(c, LC_EINVAL, "lc_distances: bad argument");
    if (!(scale > 0.0) || !std::isfinite(scale)) return fail(c, LC_ESCALE, "lc_distances: scale must be finite and > 0");
    const int L = c->nq - 1;
    const size_t N = c->N;
    const size_t Pin = (size_t)c->nq * N, Pout = (size_t)L * N;
    const int npairs = (int)(n * (n - 1) / 2);
    const bool qp = (mode & LC_HOIST_QP_SUM) != 0;
    // rotate-and-sum level: L-1 (the rescaled pair as it is) unless a level drop is asked for
    const uint32_t rl_code = (mode >> 8) & 255u;
    const int rl = rl_code ? (int)rl_code - 1 : L - 1;
    if (rl > L - 1) return fail(c, LC_ELEVEL, "lc_distances: rotation level above the rescaled level");
    const size_t Prl = (size_t)(rl + 1) * N;  // words of one output polynomial
    mode &= 1u;
    std::vector<uint32_t> sched;
    if (n_groups == 0) {
        for (int i = 1; i < c->log_n; i++) sched.push_back(1);
    } else {
        uint32_t sum = 0;
        for (uint32_t i = 0; i < n_groups; i++) {
            sched.push_back(groups ? groups[i] : 1);
            sum += sched.back();
        }
        if ((int)sum != c->log_n - 1) return fail(c, LC_EINVAL, "schedule must sum to log2(slots)");
    }
    int maxg = 1;
    for (uint32_t g : sched) maxg = std::max(maxg, (int)g);
    if (maxg > (qp ? 4 : 8)) return fail(c, LC_EINVAL, "group too large (one-ModDown groups: at most 4 bits)");
    if (!evk_usable(c, evk)) return fail(c, LC_EINVAL, "evaluation keys of a context with other parameters");
    if (!find_key(evk, -1)) return fail(c, LC_EKEY, "relinearisation key missing");
    // host buffers are staged through device memory
    const bool in_host = is_host_ptr(cts), out_host = is_host_ptr(out);
    const size_t in_words = (size_t)n * chunks * 2 * Pin, out_words = (size_t)npairs * 2 * Prl;
    const u64* din = cts;
    u64* dout = out;
    if (in_host || out_host) {
        u64* sb = stage_buf(c, ((in_host ? in_words : 0) + (out_host ? out_words : 0)) * 8);
        if (!sb) return fail(c, LC_ENOMEM, "staging buffer");
        if (in_host) {
            LC_CUDA(c, cudaMemcpyAsync(sb, cts, in_words * 8, cudaMemcpyHostToDevice, c->stream));
            din = sb;
        }
        if (out_host) dout = sb + (in_host ? in_words : 0);
    }
    // per-item scratch: acc3 + ct2 + key-switch buffers + rotation outputs
    // (with a level drop the rescaled pairs wait in scratch, 2 Pout words each, before their low
    // limbs are copied out)
    const size_t per_item = 3 * Pin + 2 * Pin + std::max(ks_words(c, 1, L), rescale_words(c, 1, 2, L)) +
                            std::max<size_t>(rotsum_words(c, 1, rl, maxg, qp), 0) + (rl < L - 1 ? 2 * Pout : 0);
    const int B = mode == LC_MODE_PER_OP ? 1 : max_batch_for(c, per_item, (size_t)8 << 30 >> 3);
    const int Bw = std::min(B, npairs);
    u64* t = lc_scratch(c, per_item * Bw * 8);
    if (!t) return fail(c, LC_ENOMEM, "scratch");
    {
        const int st0 = check_launch(c, "lc_distances (set-up)");
        if (st0) return st0;
    }
    u64* acc3 = t;
    u64* ct2 = acc3 + (size_t)Bw * 3 * Pin;
    u64* yfull = ct2 + (size_t)Bw * 2 * Pin;                  // rescaled pairs before a level drop
    u64* tmp = yfull + (rl < L - 1 ? (size_t)Bw * 2 * Pout : 0);
    for (int p0 = 0; p0 < npairs; p0 += Bw) {
        const int b = std::min(Bw, npairs - p0);
        {
            // compulsory bytes: every client tile this launch touches, once, plus the outputs
            const int touched = mode == LC_MODE_PER_OP ? 2 * b : std::min((int)n, 2 * b);
            PROF(c, PROF_TENSOR, ((double)touched * chunks * 2.0 + 3.0 * b) * Pin * 8.0, (uint64_t)b,
                 mode == LC_MODE_PER_OP ? op_sq_acc_pairs(c, din, (int)n, (int)chunks, c->nq, p0, b, acc3)
                                        : op_sq_acc_tiled(c, din, (int)n, (int)chunks, c->nq, p0, b, acc3));
        }
        int st = check_launch(c, "lc_distances (tensor accumulate)");
        if (st) return st;
        u64* y = rl < L - 1 ? yfull : dout + (size_t)p0 * 2 * Prl;
        if (mode == LC_MODE_PER_OP) {  // one operation per launch sequence: relinearise, then rescale
            st = do_relin(c, evk, acc3, b, L, ct2, tmp);
            if (!st) st = check_launch(c, "lc_distances (relinearisation)");
            if (st) return st;
            do_rescale(c, ct2, b, 2, L, y, tmp);
        } else {
            st = do_relin_rescale(c, evk, acc3, b, L, y, tmp);
            if (st) return st;
        }
        st = check_launch(c, "lc_distances (relinearisation + rescale)");
        if (st) return st;
        if (rl < L - 1) {
            // level drop: the limbs q_0 .. q_rl of each of the 2b polynomials, into the output
            u64* yl = dout + (size_t)p0 * 2 * Prl;
            LC_CUDA(c, cudaMemcpy2DAsync(yl, Prl * 8, y, Pout * 8, Prl * 8, (size_t)2 * b, cudaMemcpyDeviceToDevice,
                                         c->stream));
            y = yl;
        }
        st = do_rotate_sum(c, evk, y, b, rl, (int)sched.size(), sched.data(), tmp, qp);
        if (!st) st = check_launch(c, "lc_distances (rotate-and-sum)");
        if (st) return st;
    }
    if (out_host) LC_CUDA(c, cudaMemcpyAsync(out, dout, out_words * 8, cudaMemcpyDeviceToHost, c->stream));
    if (out_scale) *out_scale = scale * scale / (double)c->mod[L];
    if (in_host || out_host) LC_CUDA(c, cudaStreamSynchronize(c->stream));
    return check_launch(c, "lc_distances");
}

// ------------------------------------------------------------------------------------ multi-job batches
}  // extern "C"
namespace {
// host-built descriptors of one wave, uploaded into the tail of the scratch arena
struct WaveBlob {
    std::vector<unsigned char> bytes;
    template <typename T>
    size_t put(const T* p, size_t n) {
        size_t off = (bytes.size() + 255) & ~(size_t)255;
        bytes.resize(off + n * sizeof(T));
        std::memcpy(bytes.data() + off, p, n * sizeof(T));
        return off;
    }
};
// (chunk and client counts are bounded far above any device memory so that the tensor kernels'
// 64-bit partial sums cannot overflow)
bool job_ok(lc_ctx* c, const lc_job& j, bool agg) {
    if (!j.evk || !j.cts || j.chunks == 0 || j.chunks >= (1u << 20) || j.n >= (1u << 21)) return false;
    if (agg) return j.n >= 1 && j.masks && j.out_agg;
    return j.n >= 2 && j.out_dist;
}
}  // namespace

// relinearisation + rescale + (optional) rotate-and-sum of `b` items whose degree-2 sums are in
// acc3, with per-item key pointer arrays already on the device; results in y [b][2][L][N]
static int items_tail(lc_ctx* c, u64* acc3, u64* y, u64* tmp, int b, const u64* const* relin_keys,
                      const std::vector<const u64* const*>& group_keys, const std::vector<int>& group_t,
                      const std::vector<std::vector<uint64_t>>& group_gal, bool rotate, bool qp) {
    const int L = c->nq - 1;
    const size_t N = c->N;
    const size_t Pin = (size_t)c->nq * N;
    {
        KsBufs kb = ks_layout(c, tmp, b, L);
        ks_modup(c, acc3 + 2 * Pin, 3 * Pin, b, L, kb);
        PROF(c, PROF_INNER, (double)N * 8.0 * b * (c->digits(L) + 2.0) * (L + 1 + c->np), (uint64_t)b,
             op_inner_items(c, kb.ext, acc3 + 2 * Pin, 3 * Pin, b, L, relin_keys, 1, kb.v, 0));
        c->n_keyswitch += (uint64_t)b;
        ks_moddown_rescale(c, kb.v, b, L, kb, acc3, 3 * Pin, acc3 + Pin, 3 * Pin, y, (size_t)2 * L * N);
    }
    if (!rotate) return check_launch(c, "batch (relinearise + rescale)");
    const int level = L - 1, nl = L, rows = nl + c->np;
    const size_t P = (size_t)nl * N;
    KsBufs kb = ks_layout(c, tmp, b, level);
    u64* wbase = tmp + ks_words(c, b, level);
    for (size_t gi = 0; gi < group_keys.size(); gi++) {
        const int cnt = group_t[gi];
        ks_modup(c, y + P, 2 * P, b, level, kb);
        if (qp && cnt > 1) {
            const size_t vsz = (size_t)b * 2 * rows * N;
            u64* usum = wbase;
            u64* c0acc = usum + vsz;
            PROF(c, PROF_INNER, inner_gather_bytes(c, b, level, cnt), (uint64_t)b,
                 op_inner_gather(c, kb.ext, y + P, 2 * P, y, 2 * P, b, level, nullptr, group_keys[gi],
                                 group_gal[gi].data(), cnt, usum, c0acc));
            c->n_keyswitch += (uint64_t)b * cnt;
            ks_moddown(c, usum, b, level, kb, c0acc, P, y + P, 2 * P, y, 2 * P);
        } else {
            // one ModDown per rotation: W_t = (y0 + MD(v_t0), MD(v_t1)) in the pre-permuted frame
            const size_t vsz = (size_t)b * 2 * rows * N;
            u64* vs = wbase;                             // [cnt][b][2][rows][N]
            u64* ws = vs + (size_t)cnt * vsz;            // [cnt][b][2][nl][N]
            PROF(c, PROF_INNER, (double)N * 8.0 * b * (c->digits(level) + 2.0 * cnt) * rows, (uint64_t)b,
                 op_inner_items(c, kb.ext, y + P, 2 * P, b, level, group_keys[gi], cnt, vs, vsz));
            c->n_keyswitch += (uint64_t)b * cnt;
            for (int t = 0; t < cnt; t++)
                ks_moddown(c, vs + (size_t)t * vsz, b, level, kb, y, 2 * P, nullptr, 0, ws + (size_t)t * b * 2 * P,
                           2 * P);
            for (int t = 0; t < cnt; t++)
                PROF(c, PROF_AUTO, (double)b * 2 * P * 8.0 * 3.0, (uint64_t)b,
                     op_gather(c, ws + (size_t)t * b * 2 * P, y, b * 2, nl, group_gal[gi][t], true));
        }
    }
    return check_launch(c, "batch (rotate-and-sum)");
}

extern "C" {

int lc_batch_distances(lc_ctx* c, const lc_job* jobs, uint32_t n_jobs, uint32_t flags, uint32_t n_groups,
                       const uint32_t* groups) {
    if (!c || (!jobs && n_jobs)) return fail(c, LC_EINVAL, "lc_batch_distances: bad argument");
    clear_prior_error();
    const int L = c->nq - 1;
    const size_t N = c->N;
    const size_t Pin = (size_t)c->nq * N, Pout = (size_t)L * N;
    const bool qp = (flags & LC_HOIST_QP_SUM) != 0;
    std::vector<uint32_t> sched;
    if (n_groups == 0) {
        for (int i = 1; i < c->log_n; i++) sched.push_back(1);
    } else {
        uint32_t sum = 0;
        for (uint32_t i = 0; i < n_groups; i++) {
            sched.push_back(groups ? groups[i] : 1);
            sum += sched.back();
        }
        if ((int)sum != c->log_n - 1) return fail(c, LC_EINVAL, "schedule must sum to log2(slots)");
    }
    int maxg = 1;
    for (uint32_t g : sched) maxg = std::max(maxg, (int)g);
    if (maxg > 4) return fail(c, LC_EINVAL, "batched groups are limited to size 4");
    const size_t rot_words = std::max<size_t>(rotsum_words(c, 1, L - 1, maxg, qp),
                                              ks_words(c, 1, L - 1) + ((((size_t)1 << maxg) - 1) * 2 * (L + c->np) +
                                                                       (((size_t)1 << maxg) - 1) * 2 * L) * N);
    const size_t per_item = 3 * Pin + 2 * Pin + 2 * Pout + std::max(ks_words(c, 1, L), rescale_words(c, 1, 2, L)) +
                            rot_words + 64;
    const int Bcap = max_batch_for(c, per_item, (size_t)8 << 30 >> 3);
    // every item: (job, pair) of the jobs that share waves; a job with at least half a wave of
    // pairs runs alone through the single-job path (keys shared by the whole launch, no
    // per-item key tables), after the shared waves
    struct It { int job, i, j, p; };
    std::vector<It> items;
    std::vector<uint32_t> alone;
    for (uint32_t jb = 0; jb < n_jobs; jb++) {
        const lc_job& J = jobs[jb];
        if (!job_ok(c, J, false)) return fail(c, LC_EINVAL, "lc_batch_distances: job " + std::to_string(jb) + " invalid");
        if (!evk_usable(c, J.evk))
            return fail(c, LC_EINVAL, "job " + std::to_string(jb) + ": evaluation keys of a context with other parameters");
        if (!find_key(J.evk, -1)) return fail(c, LC_EKEY, "job " + std::to_string(jb) + ": relinearisation key missing");
        long stride = 1;
        for (uint32_t g : sched) {
            for (int t = 1; t < (1 << g); t++)
                if (!find_key(J.evk, (int32_t)(t * stride)))
                    return fail(c, LC_EKEY, "job " + std::to_string(jb) + ": rotation key " + std::to_string(t * stride) +
                                                " missing");
            stride <<= g;
        }
        if ((uint64_t)J.n * (J.n - 1) / 2 >= (uint64_t)std::max(1, Bcap / 2)) {
            alone.push_back(jb);
            continue;
        }
        int p = 0;
        for (uint32_t i = 0; i < J.n; i++)
            for (uint32_t j = i + 1; j < J.n; j++) items.push_back(It{(int)jb, (int)i, (int)j, p++});
    }
    auto run_alone = [&]() {
        for (uint32_t jb : alone) {
            const lc_job& J = jobs[jb];
            const int st = lc_distances(c, J.evk, J.cts, J.n, J.chunks, 1.0, LC_MODE_BATCHED | (qp ? LC_HOIST_QP_SUM : 0),
                                        (uint32_t)sched.size(), sched.data(), J.out_dist, nullptr);
            if (st) return st;
        }
        return (int)LC_OK;
    };
    if (items.empty()) return run_alone();
    const int Bw = std::min<int>(Bcap, (int)items.size());
    const size_t desc_words = (size_t)Bw * 64 + 4096;
    u64* t = lc_scratch(c, (per_item * Bw + desc_words) * 8);
    if (!t) return fail(c, LC_ENOMEM, "scratch");
    u64* acc3 = t;
    u64* ct2 = acc3 + (size_t)Bw * 3 * Pin;
    u64* y = ct2 + (size_t)Bw * 2 * Pin;
    u64* tmp = y + (size_t)Bw * 2 * Pout;
    unsigned char* desc = reinterpret_cast<unsigned char*>(t + per_item * Bw);
    for (size_t w0 = 0; w0 < items.size(); w0 += Bw) {
        const int b = (int)std::min<size_t>(Bw, items.size() - w0);
        WaveBlob blob;
        std::vector<const u64*> rk(b);
        std::vector<u64*> dst(b);
        std::vector<std::vector<const u64*>> gk(sched.size(), std::vector<const u64*>());
        std::vector<std::vector<uint64_t>> gal(sched.size());
        std::vector<int> gt(sched.size());
        for (int k = 0; k < b; k++) {
            const It& it = items[w0 + k];
            const lc_job& J = jobs[it.job];
            rk[k] = find_key(J.evk, -1)->data;
            dst[k] = J.out_dist + (size_t)it.p * 2 * Pout;
            long stride = 1;
            for (size_t gi = 0; gi < sched.size(); gi++) {
                const int cnt = (1 << sched[gi]) - 1;
                gt[gi] = cnt;
                for (int tt = 1; tt <= cnt; tt++) {
                    const SwKey* key = find_key(J.evk, (int32_t)(tt * stride));
                    // the one-ModDown group kernel reads the group-kernel layout
                    gk[gi].push_back(qp && cnt > 1 ? key->qp : key->data);
                    if (k == 0) gal[gi].push_back(key->galois);
                }
                stride <<= sched[gi];
            }
        }
        const size_t o_rk = blob.put(rk.data(), rk.size());
        const size_t o_dst = blob.put(dst.data(), dst.size());
        std::vector<size_t> o_gk(sched.size());
        for (size_t gi = 0; gi < sched.size(); gi++) o_gk[gi] = blob.put(gk[gi].data(), gk[gi].size());
        if (blob.bytes.size() > desc_words * 8) return fail(c, LC_EINVAL, "descriptor area too small");
        LC_CUDA(c, cudaMemcpyAsync(desc, blob.bytes.data(), blob.bytes.size(), cudaMemcpyHostToDevice, c->stream));
        // tensor phase: the wave's items are runs of consecutive pairs of one job each; every run
        // takes the client-block-tiled kernel of that job (each client tile read about n/8 times
        // instead of once per pair it belongs to)
        for (int k0 = 0; k0 < b;) {
            const It& first = items[w0 + k0];
            int k1 = k0 + 1;
            while (k1 < b && items[w0 + k1].job == first.job && items[w0 + k1].p == first.p + (k1 - k0)) k1++;
            const lc_job& J = jobs[first.job];
            const double touched = std::min<double>(J.n, 2.0 * (k1 - k0));
            PROF(c, PROF_TENSOR, (touched * J.chunks * 2.0 + 3.0 * (k1 - k0)) * Pin * 8.0, (uint64_t)(k1 - k0),
                 op_sq_acc_tiled(c, J.cts, (int)J.n, (int)J.chunks, c->nq, first.p, k1 - k0,
                                 acc3 + (size_t)k0 * 3 * Pin));
            k0 = k1;
        }
        std::vector<const u64* const*> gkd(sched.size());
        for (size_t gi = 0; gi < sched.size(); gi++) gkd[gi] = reinterpret_cast<const u64* const*>(desc + o_gk[gi]);
        int st = items_tail(c, acc3, y, tmp, b, reinterpret_cast<const u64* const*>(desc + o_rk), gkd, gt, gal,
                            true, qp);
        if (st) return st;
        op_copy_items(c, y, 2 * Pout, reinterpret_cast<u64* const*>(desc + o_dst), b);
        // the next wave rewrites the descriptors: wait until this wave has consumed them
        LC_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    const int st = run_alone();
    if (st) return st;
    return check_launch(c, "lc_batch_distances");
}

int lc_batch_aggregate(lc_ctx* c, const lc_job* jobs, uint32_t n_jobs) {
    if (!c || (!jobs && n_jobs)) return fail(c, LC_EINVAL, "lc_batch_aggregate: bad argument");
    clear_prior_error();
    const int L = c->nq - 1;
    const size_t N = c->N;
    const size_t Pin = (size_t)c->nq * N, Pout = (size_t)L * N;
    const size_t per_item = 3 * Pin + 2 * Pin + 2 * Pout + std::max(ks_words(c, 1, L), rescale_words(c, 1, 2, L)) + 64;
    const int Bcap = max_batch_for(c, per_item, (size_t)8 << 30 >> 3);
    // chunks of the jobs that share waves; a job with at least half a wave of chunks runs alone
    // through the single-job path after the shared waves
    struct It { int job, k; };
    std::vector<It> items;
    std::vector<uint32_t> alone;
    for (uint32_t jb = 0; jb < n_jobs; jb++) {
        const lc_job& J = jobs[jb];
        if (!job_ok(c, J, true)) return fail(c, LC_EINVAL, "lc_batch_aggregate: job " + std::to_string(jb) + " invalid");
        if (!evk_usable(c, J.evk))
            return fail(c, LC_EINVAL, "job " + std::to_string(jb) + ": evaluation keys of a context with other parameters");
        if (!find_key(J.evk, -1)) return fail(c, LC_EKEY, "job " + std::to_string(jb) + ": relinearisation key missing");
        if (J.chunks >= (uint32_t)std::max(1, Bcap / 2)) {
            alone.push_back(jb);
            continue;
        }
        for (uint32_t k = 0; k < J.chunks; k++) items.push_back(It{(int)jb, (int)k});
    }
    auto run_alone = [&]() {
        for (uint32_t jb : alone) {
            const lc_job& J = jobs[jb];
            const int st = lc_masked_aggregate(c, J.evk, J.cts, J.n, J.chunks, 1.0, J.masks, 1.0, LC_MODE_BATCHED,
                                               J.out_agg, nullptr);
            if (st) return st;
        }
        return (int)LC_OK;
    };
    if (items.empty()) return run_alone();
    const int Bw = std::min<int>(Bcap, (int)items.size());
    const size_t desc_words = (size_t)Bw * 16 + 1024;
    u64* t = lc_scratch(c, (per_item * Bw + desc_words) * 8);
    if (!t) return fail(c, LC_ENOMEM, "scratch");
    u64* acc3 = t;
    u64* ct2 = acc3 + (size_t)Bw * 3 * Pin;
    u64* y = ct2 + (size_t)Bw * 2 * Pin;
    u64* tmp = y + (size_t)Bw * 2 * Pout;
    unsigned char* desc = reinterpret_cast<unsigned char*>(t + per_item * Bw);
    for (size_t w0 = 0; w0 < items.size(); w0 += Bw) {
        const int b = (int)std::min<size_t>(Bw, items.size() - w0);
        WaveBlob blob;
        std::vector<AggItem> ai(b);
        std::vector<const u64*> rk(b);
        std::vector<u64*> dst(b);
        for (int k = 0; k < b; k++) {
            const It& it = items[w0 + k];
            const lc_job& J = jobs[it.job];
            ai[k] = AggItem{J.cts, J.masks, (int)J.n, (int)J.chunks, it.k, k};
            rk[k] = find_key(J.evk, -1)->data;
            dst[k] = J.out_agg + (size_t)it.k * 2 * Pout;
        }
        const size_t o_items = blob.put(ai.data(), ai.size());
        const size_t o_rk = blob.put(rk.data(), rk.size());
        const size_t o_dst = blob.put(dst.data(), dst.size());
        if (blob.bytes.size() > desc_words * 8) return fail(c, LC_EINVAL, "descriptor area too small");
        LC_CUDA(c, cudaMemcpyAsync(desc, blob.bytes.data(), blob.bytes.size(), cudaMemcpyHostToDevice, c->stream));
        PROF(c, PROF_TENSOR, 0.0, (uint64_t)b,
             op_mask_acc_items(c, reinterpret_cast<const AggItem*>(desc + o_items), b, c->nq, acc3));
        int st = items_tail(c, acc3, y, tmp, b, reinterpret_cast<const u64* const*>(desc + o_rk), {}, {}, {},
                            false, false);
        if (st) return st;
        op_copy_items(c, y, 2 * Pout, reinterpret_cast<u64* const*>(desc + o_dst), b);
        LC_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    const int st = run_alone();
    if (st) return st;
    return check_launch(c, "lc_batch_aggregate");
}

int lc_masked_aggregate(lc_ctx* c, const lc_evk* evk, const uint64_t* cts, uint32_t n, uint32_t chunks, double scale,
                        const uint64_t* masks, double mask_scale, uint32_t mode, uint64_t* out, double* out_scale) {
    clear_prior_error();
    if (!c || !evk || !cts || !masks || !out || n == 0 || chunks == 0)
        return fail(c, LC_EINVAL, "lc_masked_aggregate: bad argument");
    if (!(scale > 0.0) || !std::isfinite(scale) || !(mask_scale > 0.0) || !std::isfinite(mask_scale))
        return fail(c, LC_ESCALE, "lc_masked_aggregate: scales must be finite and > 0");
    const int L = c->nq - 1;
    const size_t N = c->N;
    const size_t Pin = (size_t)c->nq * N, Pout = (size_t)L * N;
    if (!evk_usable(c, evk)) return fail(c, LC_EINVAL, "evaluation keys of a context with other parameters");
    if (!find_key(evk, -1)) return fail(c, LC_EKEY, "relinearisation key missing");
    const bool in_host = is_host_ptr(cts), m_host = is_host_ptr(masks), out_host = is_host_ptr(out);
    const size_t in_words = (size_t)n * chunks * 2 * Pin, m_words = (size_t)n * 2 * Pin,
                 out_words = (size_t)chunks * 2 * Pout;
    const u64* din = cts;
    const u64* dm = masks;
    u64* dout = out;
    if (in_host || m_host || out_host) {
        u64* sb = stage_buf(c, ((in_host ? in_words : 0) + (m_host ? m_words : 0) + (out_host ? out_words : 0)) * 8);
        if (!sb) return fail(c, LC_ENOMEM, "staging buffer");
        u64* cur = sb;
        if (in_host) {
            LC_CUDA(c, cudaMemcpyAsync(cur, cts, in_words * 8, cudaMemcpyHostToDevice, c->stream));
            din = cur;
            cur += in_words;
        }
        if (m_host) {
            LC_CUDA(c, cudaMemcpyAsync(cur, masks, m_words * 8, cudaMemcpyHostToDevice, c->stream));
            dm = cur;
            cur += m_words;
        }
        if (out_host) dout = cur;
    }
    const size_t per_item = 3 * Pin + 2 * Pin + std::max(ks_words(c, 1, L), rescale_words(c, 1, 2, L));
    const int B = mode == LC_MODE_PER_OP ? 1 : max_batch_for(c, per_item, (size_t)8 << 30 >> 3);
    const int Bw = std::min(B, (int)chunks);
    u64* t = lc_scratch(c, per_item * Bw * 8);
    if (!t) return fail(c, LC_ENOMEM, "scratch");
    u64* acc3 = t;
    u64* ct2 = acc3 + (size_t)Bw * 3 * Pin;
    u64* tmp = ct2 + (size_t)Bw * 2 * Pin;
    for (int k0 = 0; k0 < (int)chunks; k0 += Bw) {
        const int b = std::min(Bw, (int)chunks - k0);
        PROF(c, PROF_TENSOR, ((double)n * b * 2.0 + 2.0 * n + 3.0 * b) * Pin * 8.0, (uint64_t)b,
             op_mask_acc(c, din, (int)n, (int)chunks, c->nq, dm, k0, b, acc3));
        int st;
        if (mode == LC_MODE_PER_OP) {
            st = do_relin(c, evk, acc3, b, L, ct2, tmp);
            if (st) return st;
            do_rescale(c, ct2, b, 2, L, dout + (size_t)k0 * 2 * Pout, tmp);
        } else {
            st = do_relin_rescale(c, evk, acc3, b, L, dout + (size_t)k0 * 2 * Pout, tmp);
            if (st) return st;
        }
    }
    if (out_host) LC_CUDA(c, cudaMemcpyAsync(out, dout, out_words * 8, cudaMemcpyDeviceToHost, c->stream));
    if (out_scale) *out_scale = scale * mask_scale / (double)c->mod[L];
    if (in_host || m_host || out_host) LC_CUDA(c, cudaStreamSynchronize(c->stream));
    return check_launch(c, "lc_masked_aggregate");
}

}  // extern "C"

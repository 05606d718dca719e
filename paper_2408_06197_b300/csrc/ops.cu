// Evaluation kernels of the Lancelot server path (elementwise RNS arithmetic, tensor and
// lazy accumulation, base conversion, key inner product, rescale, automorphism).
#include <cuda_runtime.h>
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

// grid: x = chunk (fastest; the masks are shared by every chunk), y = tile, z = limb
__global__ void __launch_bounds__(kT) k_mask_acc(const u64* __restrict__ cts, int n, int chunks, int nl, int log_n,
                                                 int k0, const u64* __restrict__ masks,
                                                 const ModConst* __restrict__ mc, u64* __restrict__ out) {
    const int k = k0 + blockIdx.x;
    const int limb = blockIdx.z;
    const size_t x = (size_t)blockIdx.y * kT + threadIdx.x;
    const size_t N = (size_t)1 << log_n;
    const ModConst m = mc[limb];
    const size_t P = (size_t)nl * N;
    u128v s00{0, 0}, s01{0, 0}, s11{0, 0};
    for (int i = 0; i < n; i++) {
        const u64* a = cts + ((size_t)i * chunks + k) * 2 * P + (size_t)limb * N + x;
        const u64* w = masks + (size_t)i * 2 * P + (size_t)limb * N + x;
        const u64 a0 = __ldg(a), a1 = __ldg(a + P), m0 = __ldg(w), m1 = __ldg(w + P);
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
    u64* o = out + (size_t)blockIdx.x * 3 * P + (size_t)limb * N + x;
    o[0] = reduce128(s00, m);
    o[P] = reduce128(s01, m);
    o[2 * P] = reduce128(s11, m);
}

// ---------------------------------------------------------------------------- base conversion
// grid: x = coefficient tile, y = b * beta + j
__global__ void __launch_bounds__(kT) k_modup(const u64* __restrict__ coef, size_t coef_stride, int beta, int rows,
                                              int log_n, const ModUpTab* __restrict__ tabs,
                                              const ModConst* __restrict__ mc, u64* __restrict__ ext) {
    __shared__ ModUpTab tab;
    const int b = blockIdx.y / beta, j = blockIdx.y - b * beta;
    {
        const int words = sizeof(ModUpTab) / 8;
        const u64* src = reinterpret_cast<const u64*>(tabs + j);
        u64* dst = reinterpret_cast<u64*>(&tab);
        for (int w = threadIdx.x; w < words; w += blockDim.x) dst[w] = src[w];
    }
    __syncthreads();
    const size_t N = (size_t)1 << log_n;
    const size_t x = (size_t)blockIdx.x * kT + threadIdx.x;
    const u64* cb = coef + (size_t)b * coef_stride + x;
    u64 y[LC_MAX_SRC];
    bool neg[LC_MAX_SRC];
    const int ns = tab.n_src;
#pragma unroll
    for (int i = 0; i < LC_MAX_SRC; i++) {
        if (i < ns) {
            const u64 q = tab.src_q[i];
            const u64 v = __ldg(cb + ((size_t)tab.src_row[i] << log_n));
            y[i] = csub(mul_shoup_lazy(v, tab.hinv[i], tab.hinv_sh[i], q), q);
            neg[i] = y[i] > (q >> 1);
        }
    }
    u64* eb = ext + ((size_t)b * beta + j) * rows * N + x;
    for (int t = 0; t < tab.n_dst; t++) {
        const ModConst m = mc[tab.dst_mod[t]];
        u128v acc{0, 0};
#pragma unroll
        for (int i = 0; i < LC_MAX_SRC; i++) {
            if (i < ns) {
                mac128(acc, y[i], tab.hat[i][t]);
                if (neg[i]) {
                    const u64 cr = tab.corr[i][t];
                    acc.lo += cr;
                    acc.hi += acc.lo < cr ? 1 : 0;
                }
            }
        }
        eb[(size_t)tab.dst_row[t] << log_n] = reduce128(acc, m);
    }
}

// grid: x = batch item (fastest, so one key tile serves every item through L2), y = tile, z = row
__global__ void __launch_bounds__(kT) k_inner(const u64* __restrict__ ext, const u64* __restrict__ d, size_t d_stride,
                                              int beta, int nl, int rows, int alpha, int nq, int nqp, int log_n,
                                              const u64* __restrict__ key, const ModConst* __restrict__ mc,
                                              int mod_of_p0, u64* __restrict__ v) {
    const int b = blockIdx.x, t = blockIdx.z;
    const size_t N = (size_t)1 << log_n;
    const size_t x = (size_t)blockIdx.y * kT + threadIdx.x;
    const int kt = t < nl ? t : nq + (t - nl);
    const ModConst m = mc[t < nl ? t : mod_of_p0 + (t - nl)];
    u128v a0{0, 0}, a1{0, 0};
    for (int j = 0; j < beta; j++) {
        u64 e;
        if (t < nl && t / alpha == j) e = __ldg(d + (size_t)b * d_stride + ((size_t)t << log_n) + x);
        else e = __ldg(ext + (((size_t)b * beta + j) * rows + t) * N + x);
        const u64 kb = __ldg(key + (((size_t)j * 2 + 0) * nqp + kt) * N + x);
        const u64 ka = __ldg(key + (((size_t)j * 2 + 1) * nqp + kt) * N + x);
        mac128(a0, e, kb);
        mac128(a1, e, ka);
    }
    u64* vb = v + (size_t)b * 2 * rows * N + (size_t)t * N + x;
    vb[0] = reduce128(a0, m);
    vb[(size_t)rows * N] = reduce128(a1, m);
}

// grid: x = tile, y = b * 2 + k
__global__ void __launch_bounds__(kT) k_moddown_bconv(const u64* __restrict__ v, int nl, int rows, int log_n,
                                                      const ModDownTab* __restrict__ tabp,
                                                      const ModConst* __restrict__ mc, u64* __restrict__ conv) {
    __shared__ ModDownTab tab;
    {
        const int words = sizeof(ModDownTab) / 8;
        const u64* src = reinterpret_cast<const u64*>(tabp);
        u64* dst = reinterpret_cast<u64*>(&tab);
        for (int w = threadIdx.x; w < words; w += blockDim.x) dst[w] = src[w];
    }
    __syncthreads();
    const size_t N = (size_t)1 << log_n;
    const size_t x = (size_t)blockIdx.x * kT + threadIdx.x;
    const int bk = blockIdx.y;
    const u64* vb = v + (size_t)bk * rows * N + x;
    const int K = tab.K;
    u64 y[LC_MAX_P];
    bool neg[LC_MAX_P];
#pragma unroll
    for (int k = 0; k < LC_MAX_P; k++) {
        if (k < K) {
            const u64 p = tab.p[k];
            const u64 val = __ldg(vb + ((size_t)(nl + k) << log_n));
            y[k] = csub(mul_shoup_lazy(val, tab.phinv[k], tab.phinv_sh[k], p), p);
            neg[k] = y[k] > (p >> 1);
        }
    }
    u64* cb = conv + (size_t)bk * nl * N + x;
    for (int i = 0; i < nl; i++) {
        const ModConst m = mc[i];
        u128v acc{0, 0};
#pragma unroll
        for (int k = 0; k < LC_MAX_P; k++) {
            if (k < K) {
                mac128(acc, y[k], tab.phat[k][i]);
                if (neg[k]) {
                    const u64 cr = tab.corr[k][i];
                    acc.lo += cr;
                    acc.hi += acc.lo < cr ? 1 : 0;
                }
            }
        }
        cb[(size_t)i << log_n] = reduce128(acc, m);
    }
}

__global__ void k_moddown_combine(const u64* __restrict__ v, const u64* __restrict__ conv, int B, int nl, int rows,
                                  int log_n, const ModDownTab* __restrict__ tab, const ModConst* __restrict__ mc,
                                  const u64* __restrict__ add0, const u64* __restrict__ add1, size_t add_stride,
                                  u64* __restrict__ w, size_t w_stride) {
    const size_t N = (size_t)1 << log_n;
    const size_t total = (size_t)B * 2 * nl * N;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
        const size_t x = idx & (N - 1);
        const size_t r = idx >> log_n;  // (b*2 + k)*nl + i
        const int i = (int)(r % nl);
        const size_t bk = r / nl;
        const int k = (int)(bk & 1);
        const size_t b = bk >> 1;
        const ModConst m = mc[i];
        const u64 vv = v[(bk * rows + i) * N + x];
        const u64 cc = conv[(bk * nl + i) * N + x];
        u64 o = mul_shoup(sub_mod(vv, cc, m.q), tab->pinv[i], tab->pinv_sh[i], m.q);
        const u64* add = k == 0 ? add0 : add1;
        if (add) o = add_mod(o, add[b * add_stride + ((size_t)i << log_n) + x], m.q);
        w[b * w_stride + ((size_t)(k * nl + i) << log_n) + x] = o;
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
__global__ void k_gather(const u64* __restrict__ w, u64* __restrict__ y, int n_polys, int nl, int log_n, uint64_t g,
                         const ModConst* __restrict__ mc, int accumulate) {
    const size_t N = (size_t)1 << log_n;
    const size_t total = (size_t)n_polys * nl * N;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
        const unsigned x = (unsigned)(idx & (N - 1));
        const size_t row = idx >> log_n;
        const u64 val = w[(row << log_n) + auto_src(x, g, log_n)];
        if (accumulate) {
            const int i = (int)(row % nl);
            y[idx] = add_mod(y[idx], val, mc[i].q);
        } else {
            y[idx] = val;
        }
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

void op_mask_acc(lc_ctx* c, const u64* cts, int n, int chunks, int nl, const u64* masks, int k0, int nk, u64* out) {
    dim3 grid(nk, (unsigned)(c->N / kT), nl);
    k_mask_acc<<<grid, kT, 0, c->stream>>>(cts, n, chunks, nl, c->log_n, k0, masks, c->mc, out);
    g_lc_launches += 1;
}

void op_modup(lc_ctx* c, const u64* coef, size_t coef_stride, int B, int level, u64* ext) {
    const int beta = c->digits(level);
    const int rows = level + 1 + c->np;
    dim3 grid((unsigned)(c->N / kT), B * beta);
    k_modup<<<grid, kT, 0, c->stream>>>(coef, coef_stride, beta, rows, c->log_n, c->modup + (size_t)level * c->dnum,
                                        c->mc, ext);
    g_lc_launches += 1;
}

void op_inner(lc_ctx* c, const u64* ext, const u64* d, size_t d_stride, int B, int level, const u64* key, u64* v) {
    const int beta = c->digits(level);
    const int nl = level + 1, rows = nl + c->np;
    dim3 grid(B, (unsigned)(c->N / kT), rows);
    k_inner<<<grid, kT, 0, c->stream>>>(ext, d, d_stride, beta, nl, rows, c->alpha, c->nq, c->nq + c->np, c->log_n,
                                        key, c->mc, c->nq, v);
    g_lc_launches += 1;
}

void op_moddown_bconv(lc_ctx* c, const u64* v, int B, int level, u64* conv) {
    const int nl = level + 1, rows = nl + c->np;
    dim3 grid((unsigned)(c->N / kT), B * 2);
    k_moddown_bconv<<<grid, kT, 0, c->stream>>>(v, nl, rows, c->log_n, c->moddown, c->mc, conv);
    g_lc_launches += 1;
}

void op_moddown_combine(lc_ctx* c, const u64* v, const u64* conv, int B, int level, const u64* add0, const u64* add1,
                        size_t add_stride, u64* w, size_t w_stride) {
    const int nl = level + 1, rows = nl + c->np;
    const size_t total = (size_t)B * 2 * nl * c->N;
    k_moddown_combine<<<grid_for(total), kT, 0, c->stream>>>(v, conv, B, nl, rows, c->log_n, c->moddown, c->mc, add0,
                                                             add1, add_stride, w, w_stride);
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
    k_gather<<<grid_for(total), kT, 0, c->stream>>>(w, y, n_polys, nl, c->log_n, g, c->mc, accumulate ? 1 : 0);
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

// Launchers of the evaluation kernels (ops.cu).  All pointers are device pointers; all
// layouts are [count][poly][limb][N] words, evaluation domain unless stated.
#pragma once
#include "context.cuh"

// out = a +/- b over n_polys polynomials of nl limbs (limb i mod q_i)
void op_addsub(lc_ctx* c, const u64* a, const u64* b, u64* out, int n_polys, int nl, bool sub);
// out[3] = tensor of one pair of degree-1 ciphertexts
void op_tensor(lc_ctx* c, const u64* a, const u64* b, u64* out, int nl);
// distances tensor phase: out[p] = sum_k (ct_i[k]-ct_j[k])^2 for pairs p in [p0, p0+np)
void op_sq_acc_pairs(lc_ctx* c, const u64* cts, int n, int chunks, int nl, int p0, int np, u64* out);
// same as op_sq_acc_pairs with client-block tiling (batched form): all pairs in [p0, p0+np)
void op_sq_acc_tiled(lc_ctx* c, const u64* cts, int n, int chunks, int nl, int p0, int np, u64* out);
// aggregate tensor phase: out[k] = sum_i ct_i[k] (x) M_i for chunks k in [k0, k0+nk)
void op_mask_acc(lc_ctx* c, const u64* cts, int n, int chunks, int nl, const u64* masks, int k0, int nk, u64* out);

// Hybrid key switching pieces (B polynomials at level `level`):
//  d: [B] input polys (evaluation domain, nl rows), stride d_stride words
//  scratch layout is owned by the caller (see capi.cu)
void op_modup(lc_ctx* c, const u64* coef, size_t coef_stride, int B, int level, u64* ext);
// fused ModDown + rescale (relinearisation followed by a rescale): preparation in the
// coefficient domain (z overwrites conv rows i < level) and the evaluation-domain combination
void op_mdrs_prep(lc_ctx* c, const u64* v, const u64* al, u64* conv, int B, int level);
void op_mdrs_combine(lc_ctx* c, const u64* v, const u64* z, int B, int level, const u64* add0, size_t add0_stride,
                     const u64* add1, size_t add1_stride, u64* out, size_t out_stride);
void op_inner(lc_ctx* c, const u64* ext, const u64* d, size_t d_stride, int B, int level, const u64* key, u64* v);
// inner products of one hoisted group's T keys (T <= 7), reading the extended digits once:
// v + t * v_key_stride receives [B][2][rows][N] for key t
void op_inner_multi(lc_ctx* c, const u64* ext, const u64* d, size_t d_stride, int B, int level, const u64* const* keys,
                    int T, u64* v, size_t v_key_stride);
// usum = sum_t phi_{g_t}(src_t) over n_polys polys of Q_l U P rows (src_t = src + t * src_stride)
void op_gather_sum_qp(lc_ctx* c, const u64* src, size_t src_stride, u64* usum, int n_polys, int nl,
                      const uint64_t* gs, int T);
// one hoisted group (T <= 7 rotations, one ModDown), fused inner products + automorphisms:
// usum [B][2][rows][N] = sum_t phi_{g_t}(<E, key_t>), c0acc [B][nl][N] = y0 + sum_t phi_{g_t}(y0).
// Keys: host array keys[t] shared by all items, or (keys == null) device table keys_dev[b * T + t].
void op_inner_gather(lc_ctx* c, const u64* ext, const u64* d, size_t d_stride, const u64* y0, size_t y0_stride, int B,
                     int level, const u64* const* keys, const u64* const* keys_dev, const uint64_t* gs, int T,
                     u64* usum, u64* c0acc);
void op_moddown_bconv(lc_ctx* c, const u64* v, int B, int level, u64* conv);
// W[b][k] = (v_k - conv_k) P^-1 + add_k  (add pointers may be null; per-item strides in words)
void op_moddown_combine(lc_ctx* c, const u64* v, const u64* conv, int B, int level, const u64* add0,
                        size_t add0_stride, const u64* add1, size_t add1_stride, u64* w, size_t w_stride);
// acc[b] += phi_g(c0 of ciphertext b) for B ciphertexts [B][2][nl][N] (acc [B][nl][N])
void op_gather_c0(lc_ctx* c, const u64* ct, u64* acc, int B, int nl, uint64_t g);
// rescale: lastc [B*deg][N] coefficient-domain copy of the last limb; r scratch [B*deg][level][N]
void op_rescale_prep(lc_ctx* c, const u64* lastc, int Bdeg, int level, u64* r);
void op_rescale_combine(lc_ctx* c, const u64* ct, const u64* r, int B, int deg, int level, u64* out);
// y[p][i][idx] (+)= w[p][i][perm_g(idx)] over n_polys polys of nl limbs
void op_gather(lc_ctx* c, const u64* w, u64* y, int n_polys, int nl, uint64_t g, bool accumulate);
// same over polys of Q_l U P rows (nl q rows then the special-prime rows)
void op_gather_qp(lc_ctx* c, const u64* w, u64* y, int n_polys, int nl, uint64_t g, bool accumulate);
// per-row permutation (any rows, all of length N)
void op_permute_rows(lc_ctx* c, const u64* in, u64* out, int rows, uint64_t g);
// signed integers -> residues for rows with modulus indices mods[0..nrows)
void op_to_rns_i64(lc_ctx* c, const int64_t* x, int B, const int* mods_host, int nrows, u64* out);
void op_to_rns_i32(lc_ctx* c, const int32_t* x, int B, const int* mods_host, int nrows, u64* out);
void op_to_rns_i8(lc_ctx* c, const int8_t* x, int B, const int* mods_host, int nrows, u64* out);
// b = e - a s (+ addmul * st when addmul_host[row] != 0); rows with modulus index mods
void op_key_combine(lc_ctx* c, const u64* a, const u64* s, const u64* e, const u64* st, const u64* addmul_host,
                    const int* mods_host, int nrows, u64* b_out);
// out0 = m + r u0 + e0, out1 = r u1 + e1 over nl limbs, B ciphertexts
void op_enc_combine(lc_ctx* c, const u64* m, const u64* r, const u64* e0, const u64* e1, const u64* pk, int B,
                    int nl, u64* out);
// acc = sum_p ct[p] s^p over nl limbs
void op_dec_combine(lc_ctx* c, const u64* ct, const u64* s, int deg, int nl, u64* out);
// elementwise square (evaluation domain), nl rows of modulus index = row
void op_square_rows(lc_ctx* c, const u64* s, u64* out, const int* mods_host, int nrows);

// ------------------------------------------------------------------ multi-job (ragged) batches
// one chunk k of one job: the job's ciphertexts ([n][chunks][2][nl][N]) and masks ([n][2][nl][N])
struct AggItem {
    const u64* cts;
    const u64* masks;
    int n;
    int chunks;
    int k;
    int slot;
};
void op_mask_acc_items(lc_ctx* c, const AggItem* items_dev, int count, int nl, u64* out);
// inner products with per-item keys: keys_dev[b * T + t] is item b's key for slot t
void op_inner_items(lc_ctx* c, const u64* ext, const u64* d, size_t d_stride, int B, int level,
                    const u64* const* keys_dev, int T, u64* v, size_t v_key_stride);
// dst_dev[b] <- src + b * words (words per item)
void op_copy_items(lc_ctx* c, const u64* src, size_t words, u64* const* dst_dev, int B);
// KGC step: read-out values (centred residue mod q0 / scale) and Krum / Multi-Krum selection
void op_readout_finish(lc_ctx* c, const u64* res, int count, double scale, double* out);
void op_krum(lc_ctx* c, const double* d, int n, int f, int l, int average, double* w, int* sel);
// FP64 encode of count slot vectors (log_n = 15 only: 2N = 256 x 256), see ops.cu
void op_encode(lc_ctx* c, const double* z, int count, double scale, const unsigned* pos, const double2* w256,
               const double2* wbig, double2* A, int64_t* m);
// group-kernel key layout (SwKey::qp) of `words` key words
void op_pack_key(lc_ctx* c, const u64* in, u64* out, size_t words);
// device randomness (Philox4x64-10): r, e0, e1 [count][N] of ciphertexts first .. first+count-1
void op_sample_enc(lc_ctx* c, u64 seed, u64 first, int count, int8_t* r, int32_t* e0, int32_t* e1);
// constant-slot plaintexts m[b] = (round(w[b] scale), 0, ..., 0), [count][N]
void op_const_plain(lc_ctx* c, const double* w, int count, double scale, int64_t* m);
// coefficient 0 (mod q0) of c0 + c1 s for `count` ciphertexts (stride ct_stride words), s0 = s in
// the evaluation domain of limb 0
void op_const_coef0(lc_ctx* c, const u64* cts, size_t ct_stride, int count, const u64* s0, u64* out);


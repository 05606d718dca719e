/*
 * lancelot.h -- C ABI of the B300 (sm_103a) Lancelot server evaluation library.
 *
 * The library computes, on one GPU, the server side of "Lancelot" (arXiv 2408.06197):
 * RNS-CKKS encrypted pairwise squared distances between client model updates
 * (Algorithm 1, "Server Executes": HSub, HSquare, lazy relinearisation, rescale,
 * rotate-and-sum with hoisted rotations) and the masked aggregate of the updates
 * (Algorithm 1, "ServerUpdate", with the mask of Section "Masked-based Encrypted Sorting").
 * Key generation, encryption and decryption (Section "CKKS Scheme Description") are
 * provided for the key generation center and the clients.
 *
 * Conventions
 *  - Every call returns an int status: LC_OK (0) or a negative LC_E* code.  No call aborts,
 *    exits or traps; lc_last_error() gives a one-line message for the last failure on a ctx.
 *  - Device work is asynchronous on the context's CUDA stream; lc_sync() waits and reports
 *    deferred device errors.  A context is used by one host thread at a time.
 *  - Ciphertext buffers are plain pointers in the layout [poly][limb][N] of uint64 words,
 *    limb i holding the residues mod q_i, in the library's evaluation ("NTT") domain.
 *    Every word is a canonical residue in [0, q_i); the kernels rely on it (words outside
 *    that range give unspecified results, never a fault).
 *    Batches are contiguous: [count][poly][limb][N].  Unless a parameter says "host or
 *    device", pointers to ciphertext words are device pointers owned by the caller.
 *    The canonical interchange form is the COEFFICIENT domain (lc_to_coeff / lc_to_eval):
 *    it does not depend on the transform's root of unity or ordering.
 *  - Scales are tracked by the caller (double); each evaluation call documents the
 *    resulting scale.
 *  - Randomness (secret, errors, uniform "a" polynomials, encryption ephemerals) is supplied
 *    by the caller, so that results are reproducible bit for bit; the seeded calls
 *    (lc_sample_enc, lc_encrypt_seeded, ...) instead draw it on the device from a seed
 *    (Philox4x64-10), equally reproducible.
 *  - Host transfers may use the wire form (lc_pack / lc_unpack: each residue in as many bytes
 *    as its prime needs).  Device waits are bounded; one that runs out is reported by the next
 *    lc_sync as LC_ETIMEOUT.
 */
#ifndef LANCELOT_H
#define LANCELOT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LC_OK 0
#define LC_EINVAL (-1)   /* bad argument, size or layout */
#define LC_ELEVEL (-2)   /* ciphertext level not valid for the call */
#define LC_ESCALE (-3)   /* scale mismatch */
#define LC_ENOMEM (-4)   /* allocation failed */
#define LC_ECUDA (-5)    /* CUDA runtime error (message in lc_last_error) */
#define LC_ETIMEOUT (-6) /* a bounded device wait gave up */
#define LC_EBUSY (-7)    /* resource in use */
#define LC_EKEY (-8)     /* required evaluation key missing */

typedef struct lc_ctx lc_ctx;
typedef struct lc_evk lc_evk;

/* RNS-CKKS parameters (Section "CKKS Scheme Description"): ring Z_Q[X]/(X^N+1) with
 * N = 2^log_n (12 <= log_n <= 16), Q = q_0 ... q_L (n_q = L+1 limbs), special modulus
 * P = p_0 ... p_{K-1} (n_p = K), dnum decomposition digits at level L, digit size
 * alpha = ceil((L+1)/dnum).  Every prime is < 2^62 and = 1 mod 2N.  Arrays are copied. */
typedef struct {
    uint32_t log_n;
    uint32_t n_q;
    uint32_t n_p;
    uint32_t dnum;
    const uint64_t* q;
    const uint64_t* p;
} lc_params;

/* Optional device allocator (e.g. PyTorch's caching allocator).  alloc returns a device
 * pointer of at least `bytes` (256-byte aligned) or NULL; free releases it.  With a NULL
 * allocator the library uses cudaMalloc / cudaFree. */
typedef struct {
    void* (*alloc)(size_t bytes, void* user);
    void (*free)(void* ptr, void* user);
    void* user;
} lc_allocator;

/* Evaluation modes of lc_distances / lc_masked_aggregate. */
#define LC_MODE_PER_OP 0  /* one kernel sequence per HE operation, one pair / chunk at a time */
#define LC_MODE_BATCHED 1 /* every pair / chunk in each launch, keys read once per launch */
/* Hoisting variant flag (or-ed into the mode of lc_distances, flags of lc_rotate_sum): a
 * hoisted group of rotations sums its inner products over Q_l U P and switches down once,
 * instead of once per rotation (Section "Dynamic Hoisting": the rotations of one unfolded
 * group are summed after the key switching).  Identical results for groups of size 1;
 * a different rounding (not the same bits) for larger groups. */
#define LC_HOIST_QP_SUM 2
/* Level drop before the rotate-and-sum (or-ed into the mode of lc_distances / lc_ct_distances):
 * each relinearised and rescaled pair is reduced to level l (its limbs q_0 .. q_l are kept, the
 * others discarded -- a ciphertext mod Q is one mod every Q' dividing Q, with the same message
 * while that message stays below Q'/2) and rotated and summed there: the rotations' key switches
 * then work on l + 1 limbs instead of L.  Outputs are at level l.  0 <= l <= L - 1; without it
 * the rotations run at level L - 1.  Different bits from the default (the ciphertexts have other
 * limbs); the decrypted distances agree within the noise. */
#define LC_ROTATE_AT_LEVEL(l) ((((uint32_t)(l)) + 1u) << 8)

/* ---------------------------------------------------------------- parameters / context */

/* The `count` largest `bits`-bit primes q = 1 mod 2^(log_n+1), after skipping `skip`,
 * descending, into out[count] (host).  The paper fixes only the bit sizes (scale 2^40,
 * Section "Baseline and Implementation details"); this is the library's deterministic rule. */
int lc_gen_primes(uint32_t log_n, uint32_t bits, uint32_t skip, uint32_t count, uint64_t* out);

/* Creates a context on `device` with all device tables (twiddles, base-conversion and
 * rescale constants).  `stream` is a cudaStream_t (NULL = legacy default stream). */
int lc_ctx_create(const lc_params* prm, int device, void* stream, const lc_allocator* alloc, lc_ctx** out);
void lc_ctx_destroy(lc_ctx* ctx);
int lc_set_stream(lc_ctx* ctx, void* stream);
int lc_sync(lc_ctx* ctx);
const char* lc_last_error(const lc_ctx* ctx);
/* Key switches and ModUps issued since the last reset (lazy relinearisation and hoisting
 * counters): out[0] = key switches, out[1] = ModUp decompositions. */
int lc_counters(lc_ctx* ctx, uint64_t* out, int reset);

/* Stream-ordered copies on the context's stream (no counterpart in the paper: the explicit
 * host<->device transfers that replace unified memory, Appendix "CPU-GPU Computation Model").
 * dst/src: device pointer on the device side; host side pageable or pinned. */
int lc_memcpy_h2d(lc_ctx* ctx, uint64_t* dst_dev, const void* src_host, size_t bytes);
int lc_memcpy_d2h(lc_ctx* ctx, void* dst_host, const uint64_t* src_dev, size_t bytes);
/* Overlapped host transfers (no counterpart in the paper).  The context keeps one copy stream
 * per direction.  lc_copy_async enqueues a copy on the stream of its direction (LC_H2D or
 * LC_D2H), ordered after all work enqueued on the context's stream so far, so a device buffer
 * that earlier calls still read is not overwritten and a result is read only once computed;
 * *ticket names the copy.  lc_copy_wait makes the context's stream wait for that copy.  Host
 * memory must be pinned for the copy to overlap with computation.  Not allowed inside a graph
 * capture (LC_EBUSY).  A ticket is consumed by its lc_copy_wait (waiting twice is LC_EINVAL) and
 * its event is reused by later copies; tickets never waited on hold one event each until
 * lc_ctx_destroy. */
#define LC_H2D 0
#define LC_D2H 1
int lc_copy_async(lc_ctx* ctx, void* dst, const void* src, size_t bytes, int dir, uint64_t* ticket);
int lc_copy_wait(lc_ctx* ctx, uint64_t ticket);
/* Kernel launches issued by the library in this process so far (*out). */
int lc_launches(uint64_t* out);
/* Per-kernel-class device timing with CUDA events on the context stream (measurement only).
 * start = 1 clears and starts recording; start = 0 stops, synchronises and writes per class
 * (0 NTT, 1 ModUp, 2 key inner product, 3 ModDown, 4 tensor/accumulate, 5 rescale,
 * 6 automorphism, 7 other) the summed milliseconds, algorithmic bytes and launches [8]. */
int lc_profile(lc_ctx* ctx, int start, double* ms, double* bytes, uint64_t* launches);

/* Caps how many pairs / chunks one batched wave of lc_distances / lc_masked_aggregate
 * processes (0 = only the 8 GiB scratch budget limits it).  Smaller waves use less scratch;
 * results are identical for every setting. */
int lc_set_max_batch(lc_ctx* ctx, uint32_t max_items);

/* Tile-shape knobs for an autotuner (no counterpart in the paper; the paper tunes nothing on
 * the GPU).  Every option computes identical results; only speed differs.  Unknown knobs or
 * options fail with LC_EINVAL and leave the setting unchanged.  Options (default first):
 *   LC_TUNE_NTT_ROW_MINB       row pass of the NTT: minimum resident 128-thread blocks, i.e. a
 *                              register cap: 5, 4, 6
 *   LC_TUNE_NTT_COL_MINB       column pass of the NTT: 8, 1 (no cap), 6, 7
 *   LC_TUNE_GROUP_SPLIT_ITEMS  one-ModDown group kernel, rows with primes below 2^40: items per
 *                              thread, 1 or 2
 *   LC_TUNE_GROUP_WIDE_ITEMS   same, other rows: 1 or 2
 *   LC_TUNE_TENSOR_WARPS       batched distance tensor (primes below 2^40): warps per block,
 *                              16 (4 pair slots per thread), 8 (8 slots) or 12 (6 slots)
 *   LC_TUNE_NTT_ROW_TMA        forward row pass: 0 = one block per tile, 1 = persistent blocks
 *                              streaming tiles through shared memory with bulk copies (TMA)
 *   LC_TUNE_GROUP_KARATSUBA    one-ModDown group kernel, rows with primes below 2^40: 1 = three
 *                              20-bit partial products per product (Karatsuba), 0 = four
 * The paper_2408_06197_b300.autotune module times the options on the caller's workload. */
#define LC_TUNE_NTT_ROW_MINB 1
#define LC_TUNE_NTT_COL_MINB 2
#define LC_TUNE_GROUP_SPLIT_ITEMS 3
#define LC_TUNE_GROUP_WIDE_ITEMS 4
#define LC_TUNE_TENSOR_WARPS 5
#define LC_TUNE_NTT_ROW_TMA 6
#define LC_TUNE_GROUP_KARATSUBA 7
int lc_set_tuning(lc_ctx* ctx, uint32_t knob, int32_t value);
int lc_get_tuning(const lc_ctx* ctx, uint32_t knob, int32_t* value);

/* Integer-pipe probes (measurement only; no counterpart in the paper).  Runs one register-
 * resident kernel of `kind` on the context's device and stream: blocks_per_sm x SM-count blocks
 * of 256 threads, each thread executing iters x 64 operations (LC_PROBE_NTT_BFLY: iters x 32
 * butterflies), and returns its device time in *ms (CUDA events) and the operations executed in
 * *ops.  Kinds: LC_PROBE_IMAD, 32-bit multiply-adds; LC_PROBE_IMAD_WIDE, 32 x 32 -> 64-bit
 * multiply-adds; LC_PROBE_NTT_BFLY, the lazy Shoup Cooley-Tukey butterfly of the transforms for
 * primes below 2^46 (the same code, twiddles in registers, no memory traffic).  The kernels read
 * no buffer and write none (one library-owned word at most); the call synchronises the stream.
 * LC_EINVAL for an unknown kind, iters == 0 or blocks_per_sm outside [1, 32]. */
#define LC_PROBE_IMAD 0
#define LC_PROBE_IMAD_WIDE 1
#define LC_PROBE_NTT_BFLY 2
int lc_alu_probe(lc_ctx* ctx, uint32_t kind, uint32_t iters, uint32_t blocks_per_sm, double* ms, double* ops);

/* Wire form of ciphertext arrays (no counterpart in the paper; a transfer format).  A record of
 * deg polynomials at `level` stores, polynomial after polynomial and limb after limb, the N
 * residues of limb i (canonical, below q_i) in w_i = ceil(bits(q_i - 1) / 8) little-endian bytes
 * each (4 <= w_i <= 8): a production ciphertext at level 14 takes 78 bytes per coefficient
 * instead of 120.  lc_wire_bytes gives the bytes of one record.  lc_pack / lc_unpack convert
 * `count` records between the word layout [count][deg][level+1][N] and the wire form, both on
 * the device (16-byte aligned device buffers; host buffers are LC_EINVAL -- copy with
 * lc_copy_async first).  Asynchronous on the context's stream.  lc_unpack checks every residue:
 * one that is not below its prime makes the next lc_sync return LC_EINVAL (the words written
 * for it are unspecified). */
int lc_wire_bytes(lc_ctx* ctx, uint32_t deg, uint32_t level, uint64_t* bytes);
int lc_pack(lc_ctx* ctx, const uint64_t* in, uint32_t count, uint32_t deg, uint32_t level, uint8_t* out);
int lc_unpack(lc_ctx* ctx, const uint8_t* in, uint32_t count, uint32_t deg, uint32_t level, uint64_t* out);

/* Self-test of the bounded device waits (no counterpart in the paper).  Kernels that stream tiles
 * with bulk copies wait on shared-memory barriers for at most a fixed number of polls; a wait that
 * runs out sets the context's device error word, which the next lc_sync reports as LC_ETIMEOUT
 * (and clears).  This call runs one block that copies 64 bytes through such a barrier and checks
 * them, then, if never_arrive != 0, waits at most max_polls polls on a barrier at which nothing
 * ever arrives.  Synchronous.  Returns LC_OK when the copy arrived intact and no wait ran out,
 * LC_ETIMEOUT when a wait ran out (the context stays usable), LC_EINVAL for max_polls == 0. */
int lc_wait_selftest(lc_ctx* ctx, int never_arrive, uint32_t max_polls);

/* CUDA-graph capture of a sequence of calls on the context's stream (no counterpart in the
 * paper; replaces per-call kernel launches with one graph launch).  Between lc_graph_begin and
 * lc_graph_end only device-pointer evaluation calls may be made; their scratch must already be
 * sized (run each call once before capturing), otherwise they fail with LC_ENOMEM.  The graph
 * replays the captured launches on the same buffers; the stream must not be the legacy default
 * stream. */
typedef struct lc_graph lc_graph;
int lc_graph_begin(lc_ctx* ctx);
int lc_graph_end(lc_ctx* ctx, lc_graph** out);
int lc_graph_launch(lc_ctx* ctx, const lc_graph* graph);
void lc_graph_free(lc_graph* graph);

/* ---------------------------------------------------------------- keys (KGC side) */

/* Public key pk = ([-a s + e]_Q, a) (Section "CKKS Scheme Description", Key generation).
 * s: host int8[N] ternary; a: host uint64[n_q][N] coefficient domain, row i in [0, q_i);
 * e: host int32[N]; pk_out: device uint64[2][n_q][N] (evaluation domain). */
int lc_pk_gen(lc_ctx* ctx, const int8_t* s, const uint64_t* a, const int32_t* e, uint64_t* pk_out);

/* An evaluation-key set belongs to the context that made it (free it before that context) and
 * may be used by any context with the same device, ring degree and moduli, e.g. contexts on
 * other streams; the evaluation calls reject keys of other parameters with LC_EINVAL. */
int lc_evk_create(lc_ctx* ctx, lc_evk** out);
void lc_evk_free(lc_evk* evk);
/* Adds one switching key to evk (Key generation, Evaluation key; hybrid form with dnum
 * digits): rotation < 0 adds the relinearisation key for s~ = s^2, rotation r >= 1 adds the
 * key for s~ = phi_{5^r}(s) used by left rotation by r slots (Section "Dynamic Hoisting").
 * Digit j, row t of Q U P: b = -a_j s + e_j + [q_t in D_j] (P mod q_t) s~, a = a_j.
 * s: host int8[N]; a: host uint64[dnum][n_q+n_p][N] coefficient domain; e: host int32[dnum][N].
 * The key is stored on the device (for rotations pre-permuted by phi^-1, see DESIGN).
 * Returns LC_EBUSY if the key already exists. */
int lc_evk_add(lc_ctx* ctx, lc_evk* evk, const int8_t* s, int32_t rotation, const uint64_t* a, const int32_t* e);
/* Copies a key back in canonical form: host uint64[dnum][2][n_q+n_p][N], coefficient domain. */
int lc_evk_export(lc_ctx* ctx, const lc_evk* evk, int32_t rotation, uint64_t* out);
/* Adds a key from that canonical form (no counterpart in the paper; checkpoint / restore of a key
 * set without the secret): `in` as lc_evk_export writes it, for the key of `rotation` (< 0:
 * relinearisation).  The key is stored exactly as lc_evk_add would store it, so results are
 * bit-identical.  LC_EINVAL if a residue is not below its prime, LC_EBUSY if the key exists.
 * Synchronous. */
int lc_evk_import(lc_ctx* ctx, lc_evk* evk, int32_t rotation, const uint64_t* in);

/* ---------------------------------------------------------------- client side */

/* CKKS.Encode (Section "Batch Encoding and Decoding"): m = round(scale * sigma^-1(pi^-1(z)))
 * for real z[len], len <= N/2 (zero padded); slot j <-> evaluation at xi^(5^j), xi = e^(i pi/N).
 * FP64 on the host; m_out: host int64[N]. */
int lc_encode(lc_ctx* ctx, const double* z, size_t len, double scale, int64_t* m_out);
/* CKKS.Decode of integer coefficients given as doubles: z_j = m(xi^(5^j)) / scale, real part.
 * m: host double[N]; z_out: host double[N/2]. */
int lc_decode(lc_ctx* ctx, const double* m, double scale, double* z_out);

/* CKKS.Enc (Section "CKKS Scheme Description", Encryption) of `count` plaintexts at level L:
 * ct = (m + r u0 + e0, r u1 + e1) mod Q.  pk: device [2][n_q][N] from lc_pk_gen;
 * m: host int64[count][N] (|m| < 2^63); r: host int8[count][N]; e0, e1: host int32[count][N];
 * out: device uint64[count][2][n_q][N]. */
int lc_encrypt(lc_ctx* ctx, const uint64_t* pk, const int64_t* m, const int8_t* r, const int32_t* e0,
               const int32_t* e1, uint32_t count, uint64_t* out);

/* Device-randomness mode (no counterpart in the paper, which leaves the sampler open): the
 * encryption randomness is drawn on the GPU from the counter-based generator Philox4x64-10
 * (Salmon et al., SC 2011) instead of being supplied by the caller.  Key (seed, 0); counter
 * (coefficient k, ciphertext index c, purpose p, 0) with p = 0 for r, 1 for e0, 2 for e1;
 * r = floor(3 (word0 >> 32) / 2^32) - 1; e = popcount(word0 mod 2^21) - popcount(word1 mod
 * 2^21) (centred binomial, eta = 21, sigma = 3.24).  Ciphertext b of a call has index
 * first + b, so disjoint index ranges give independent randomness for one seed.
 * lc_sample_enc returns the draws ([count][N] each, host memory) for checking.
 * lc_encrypt_seeded: Section "CKKS Scheme Description" Enc with these draws; m_dev = device
 * plaintexts [count][N] int64 (centred integers); out as lc_encrypt.
 * lc_encrypt_const_seeded: the same for constant-slot plaintexts (coefficient 0 =
 * round(w_dev[b] * scale), the others 0): the KGC's mask ciphertexts (Section "Masked-based
 * Encrypted Sorting").  Neither call synchronises the host, so both can be graph-captured. */
int lc_sample_enc(lc_ctx* ctx, uint64_t seed, uint64_t first, uint32_t count, int8_t* r, int32_t* e0, int32_t* e1);
/* Client-side batched encode on the GPU (FP64; N = 2^15 only, other N give LC_EINVAL): z_dev =
 * [count][N/2] real slot values (device doubles), m_dev = [count][N] integer plaintexts
 * (device int64), m = round(2/N Re FFT_2N(A)) with A[5^j mod 2N] = scale z_j -- the map of
 * lc_encode computed with a different FFT, so an integer may differ by one where the FP64 value
 * is within rounding error of a half-integer.  lc_encode_encrypt_seeded encodes and encrypts
 * with device randomness (ciphertext indices first ..) in one call: the clients' step of
 * Algorithm 1 for many clients and chunks without host arrays. */
int lc_encode_dev(lc_ctx* ctx, const double* z_dev, uint32_t count, double scale, int64_t* m_dev);
int lc_encode_encrypt_seeded(lc_ctx* ctx, const uint64_t* pk, const double* z_dev, uint32_t count, double scale,
                             uint64_t seed, uint64_t first, uint64_t* out);
int lc_encrypt_seeded(lc_ctx* ctx, const uint64_t* pk, const int64_t* m_dev, uint32_t count, uint64_t seed,
                      uint64_t first, uint64_t* out);
int lc_encrypt_const_seeded(lc_ctx* ctx, const uint64_t* pk, const double* w_dev, uint32_t count, double scale,
                            uint64_t seed, uint64_t first, uint64_t* out);

/* CKKS.Dec (Section "CKKS Scheme Description", Decryption): residues of c0 + c1 s (+ c2 s^2)
 * mod Q_level.  ct: device [deg][level+1][N] (deg 2 or 3); s: host int8[N];
 * res_out: host uint64[level+1][N], coefficient domain. */
int lc_decrypt(lc_ctx* ctx, const int8_t* s, const uint64_t* ct, uint32_t deg, uint32_t level, uint64_t* res_out);
/* KGC read-out of ciphertexts that hold one value in every slot (the rotate-and-summed
 * distances of Algorithm 1): the average of the slots, which is coefficient 0 of the plaintext
 * divided by the scale, computed from c0 + c1 s on limb q_0 only (a GPU reduction per
 * ciphertext).  Valid while |value * scale| < q_0 / 2.  s: host int8[N]; cts: device
 * [count][2][level+1][N]; out: host double[count]. */
int lc_decrypt_const(lc_ctx* ctx, const int8_t* s, const uint64_t* cts, uint32_t count, uint32_t level, double scale,
                     double* out);
/* KGC step on the device (Alg. 2 and the mask of Section "Masked-based Encrypted Sorting"; no
 * counterpart in the paper's GPU design, whose KGC runs on the host).  A resident KGC key keeps
 * the secret mod q0 on the device:
 *   lc_kgc_create: s = ternary secret [N] (host); lc_kgc_free releases it (before its context).
 *   lc_kgc_readout: as lc_decrypt_const, but the `count` values go to out_dev (device doubles)
 *                   and the host is not synchronised.
 *   lc_kgc_krum:    Krum / Multi-Krum on n <= 256 clients from pair distances dist_dev
 *                   (n(n-1)/2 doubles, i < j lexicographic): score_i = sum of the n - f - 2
 *                   smallest d(i, j); the n_select lowest scores are kept (ties to the lower
 *                   index); w_dev[i] = 1/n_select (average) or 1 for kept clients, 0 otherwise;
 *                   sel_dev = kept indices in score order.
 * With lc_encrypt_const_seeded for the masks, a whole round (distances, read-out, selection,
 * masks, aggregate) runs without a host round trip and can be captured in one graph. */
typedef struct lc_kgc lc_kgc;
int lc_kgc_create(lc_ctx* ctx, const int8_t* s, lc_kgc** out);
void lc_kgc_free(lc_kgc* kgc);
int lc_kgc_readout(lc_ctx* ctx, const lc_kgc* kgc, const uint64_t* cts, uint32_t count, uint32_t level, double scale,
                   double* out_dev);
int lc_kgc_krum(lc_ctx* ctx, const double* dist_dev, uint32_t n, uint32_t f, uint32_t n_select, int average,
                double* w_dev, int32_t* sel_dev);

/* Centred CRT of residues[level+1][N] (host) to doubles m_out[N] (host), exact big-integer. */
int lc_crt_to_double(lc_ctx* ctx, const uint64_t* res, uint32_t level, double* m_out);

/* ---------------------------------------------------------------- interchange */

/* In-place domain change of n_polys consecutive polynomials of level+1 limbs (device). */
int lc_to_coeff(lc_ctx* ctx, uint64_t* data, uint32_t n_polys, uint32_t level);
int lc_to_eval(lc_ctx* ctx, uint64_t* data, uint32_t n_polys, uint32_t level);

/* ---------------------------------------------------------------- evaluation primitives */

/* HAdd / HSub (Section "Private Distance Evaluation"): out = a +/- b mod q_i on n_polys
 * polynomials of level+1 limbs (device). */
int lc_add(lc_ctx* ctx, const uint64_t* a, const uint64_t* b, uint32_t n_polys, uint32_t level, uint64_t* out);
int lc_sub(lc_ctx* ctx, const uint64_t* a, const uint64_t* b, uint32_t n_polys, uint32_t level, uint64_t* out);
/* CKKS.Mult tensor (Appendix "Hardware Acceleration on Homomorphic Multiplication"):
 * out[3] = (a0 b0, a0 b1 + a1 b0, a1 b1); scale multiplies.  Device buffers. */
int lc_tensor(lc_ctx* ctx, const uint64_t* a, const uint64_t* b, uint32_t level, uint64_t* out);
/* Relinearisation (Section "Lazy Relinearization"): count degree-2 triples [count][3][level+1][N]
 * -> [count][2][level+1][N] via hybrid key switching with the relinearisation key. */
int lc_relin(lc_ctx* ctx, const lc_evk* evk, const uint64_t* ct3, uint32_t count, uint32_t level, uint64_t* out);
/* Rescale: drop q_level with centred rounding; [count][deg][level+1][N] -> [count][deg][level][N];
 * the scale divides by q_level. */
int lc_rescale(lc_ctx* ctx, const uint64_t* ct, uint32_t count, uint32_t deg, uint32_t level, uint64_t* out);
/* Rescale that allocates nothing (no counterpart in the paper).  Same inputs, outputs and
 * result as lc_rescale, but its scratch is a fixed 16 MiB device array built into the library
 * (2 Mi words; one production ciphertext of degree 2 at level 14 needs 983,040) instead of the
 * context's scratch arena, which lc_rescale may grow with cudaMalloc.  It is meant for callers
 * that cannot allocate at that point: a process whose device-memory budget is fully committed
 * at start-up, code running while its allocator must not be entered, or latency-sensitive
 * paths that cannot take the device synchronisation cudaMalloc / cudaFree can cause.
 *  - Calls no cudaMalloc, cudaFree or allocating routine, and creates no CUDA event (the call
 *    is left out of lc_profile's per-class timing).  Every GPU that loads the library holds the
 *    array until the process exits.
 *  - Launch failures are returned as LC_ECUDA by this call itself (as lc_rescale does), and a
 *    non-sticky error left by earlier unrelated code is cleared on entry.
 *  - The first call on a device looks up the array's device address (cudaGetSymbolAddress,
 *    with that device made current for the look-up); make that first call before any stream
 *    capture.  The address is kept for the life of the process: after cudaDeviceReset on that
 *    device (which also invalidates its contexts) do not call this entry point there again.
 *  - A request needing more than 16 MiB of scratch (count * deg * N * (level+1) words) is
 *    rejected with LC_EINVAL and a message in lc_last_error; split it into smaller calls.
 *  - All calls in the process share the one array and leave their last contents in it (nothing
 *    in it needs to start at zero): calls that may overlap on the GPU (different streams or
 *    contexts) race on it and must be serialised by the caller. */
int lc_rescale_noalloc(lc_ctx* ctx, const uint64_t* ct, uint32_t count, uint32_t deg, uint32_t level, uint64_t* out);

/* Hoisted rotations (Section "Dynamic Hoisting"): one ModUp of c1, then for each r in
 * rots[n_rot] the left rotation by r slots: out[k] = (phi(c0) + KS0, KS1),
 * out: device [n_rot][2][level+1][N]. */
int lc_rotate(lc_ctx* ctx, const lc_evk* evk, const uint64_t* ct, uint32_t level, uint32_t n_rot, const int32_t* rots,
              uint64_t* out);
/* Rotate-and-sum in place over `count` ciphertexts [count][2][level+1][N] with a hoisting
 * schedule: groups[n_groups] with sum = log2(N/2); group g with stride s does
 * y <- y + sum_{t=1}^{2^g-1} Rot_{t s}(y) from one ModUp, then s <- s 2^g.  All groups 1 is the
 * plain log-step sum.  Afterwards every slot holds the sum of all slots.  flags: 0 or
 * LC_HOIST_QP_SUM.  Group sizes: at most 8 bits, at most 4 (15 rotations) with LC_HOIST_QP_SUM
 * (LC_EINVAL beyond). */
int lc_rotate_sum(lc_ctx* ctx, const lc_evk* evk, uint64_t* cts, uint32_t count, uint32_t level, uint32_t n_groups,
                  const uint32_t* groups, uint32_t flags);

/* ---------------------------------------------------------------- the method */

/* Encrypted pairwise squared distances (Algorithm 1, "Server Executes"), for every pair i<j
 * in lexicographic order: Dis = rotate_sum(rescale(relin(sum_k (ct_i[k] - ct_j[k])^2))).
 * cts: host or device [n][chunks][2][n_q][N] at level L and scale `scale`;
 * out: host or device [n(n-1)/2][2][n_q-1][N] ([n(n-1)/2][2][l+1][N] with LC_ROTATE_AT_LEVEL(l));
 * *out_scale = scale^2 / q_L.
 * mode: LC_MODE_PER_OP or LC_MODE_BATCHED (same bits), optionally | LC_HOIST_QP_SUM and
 * | LC_ROTATE_AT_LEVEL(l) (LC_ELEVEL for l > L - 1).
 * groups: hoisting schedule as in
 * lc_rotate_sum (NULL = all ones).  evk must hold the relinearisation key and every
 * rotation key the schedule needs (else LC_EKEY); a scale that is not finite and positive is
 * LC_ESCALE. */
int lc_distances(lc_ctx* ctx, const lc_evk* evk, const uint64_t* cts, uint32_t n, uint32_t chunks, double scale,
                 uint32_t mode, uint32_t n_groups, const uint32_t* groups, uint64_t* out, double* out_scale);

/* Masked aggregate (Algorithm 1, "ServerUpdate"): for every chunk k,
 * out[k] = rescale(relin(sum_i ct_i[k] (x) M_i)), M_i the mask ciphertext of client i
 * (its selection weight in every slot, Section "Masked-based Encrypted Sorting").
 * cts: host or device [n][chunks][2][n_q][N]; masks: host or device [n][2][n_q][N];
 * out: host or device [chunks][2][n_q-1][N]; *out_scale = scale * mask_scale / q_L.  Scales
 * that are not finite and positive are LC_ESCALE. */
int lc_masked_aggregate(lc_ctx* ctx, const lc_evk* evk, const uint64_t* cts, uint32_t n, uint32_t chunks,
                        double scale, const uint64_t* masks, double mask_scale, uint32_t mode, uint64_t* out,
                        double* out_scale);

/* ---------------------------------------------------------------- multi-job (uneven) batches */

/* One aggregation round of one tenant: its evaluation keys, its clients' ciphertexts and its
 * outputs (all device pointers, layouts as in lc_distances / lc_masked_aggregate). */
typedef struct {
    const lc_evk* evk;     /* the tenant's relinearisation + rotation keys */
    const uint64_t* cts;   /* [n][chunks][2][n_q][N] at level L */
    uint32_t n;            /* clients (>= 2 for distances) */
    uint32_t chunks;       /* ciphertexts per client (ragged across jobs) */
    const uint64_t* masks; /* [n][2][n_q][N], for lc_batch_aggregate */
    uint64_t* out_dist;    /* [n(n-1)/2][2][n_q-1][N], for lc_batch_distances */
    uint64_t* out_agg;     /* [chunks][2][n_q-1][N], for lc_batch_aggregate */
} lc_job;

/* Encrypted distances of several rounds at once (Algorithm 1 "Server Executes" per job): the
 * (job, pair) items of small jobs -- different client counts, model sizes and key sets -- run
 * together in batched waves (per-item key tables); a job with at least half a wave of pairs runs
 * on its own through the lc_distances path (keys shared by the launch) after them.  Each job's
 * results are bit-identical to lc_distances on that job alone with the same schedule.  flags: 0
 * or LC_HOIST_QP_SUM; groups as in lc_rotate_sum (sizes <= 4).  Synchronises the stream between
 * shared waves (descriptors are rewritten). */
int lc_batch_distances(lc_ctx* ctx, const lc_job* jobs, uint32_t n_jobs, uint32_t flags, uint32_t n_groups,
                       const uint32_t* groups);
/* Masked aggregates of several rounds at once (Algorithm 1 "ServerUpdate" per job): chunks of
 * small jobs share waves, a job with at least half a wave of chunks runs through the
 * lc_masked_aggregate path; each job's results are bit-identical to lc_masked_aggregate on that
 * job alone. */
int lc_batch_aggregate(lc_ctx* ctx, const lc_job* jobs, uint32_t n_jobs);

/* ---------------------------------------------------------------- handles (level / scale tracked) */

/* The calls above take plain arrays whose level and scale the caller tracks.  The calls below
 * follow the roles of the paper's problem statement (Fig. 1 and Algorithm 1: the KGC generates
 * keys and decrypts, clients encrypt, the server evaluates with the evaluation keys only) with
 * handles that carry this metadata, so that a ciphertext at the wrong level or scale is rejected
 * (LC_ELEVEL / LC_ESCALE) instead of computed on.  They run the same kernels as the array calls
 * and give the same bits.  Every handle belongs to one context and must be freed before it. */

/* A device-resident array of `count` ciphertexts of one degree (number of polynomials, 1..3),
 * level and scale: device words [count][deg][level+1][N] in the evaluation domain. */
typedef struct lc_ct lc_ct;
/* The KGC's secret key (a host copy of the ternary secret) and the public key (device). */
typedef struct lc_sk lc_sk;
typedef struct lc_pk lc_pk;

/* A handle of `count` ciphertexts, all words zero (valid residues).  LC_ELEVEL for level > L,
 * LC_ESCALE for a scale that is not finite and positive. */
int lc_ct_create(lc_ctx* ctx, uint32_t count, uint32_t deg, uint32_t level, double scale, lc_ct** out);
/* Imports ciphertexts given in the canonical interchange form: host uint64
 * [count][deg][level+1][N], COEFFICIENT domain, every residue below its prime (else LC_EINVAL,
 * checked on the host before anything is copied).  Synchronous. */
int lc_ct_import(lc_ctx* ctx, const uint64_t* coeffs, uint32_t count, uint32_t deg, uint32_t level, double scale,
                 lc_ct** out);
/* Exports a handle in that form into host coeffs[count][deg][level+1][N], and its level and
 * scale (either may be NULL).  Synchronous. */
int lc_ct_export(const lc_ct* ct, uint64_t* coeffs, uint32_t* level, double* scale);
/* Metadata of a handle (any output may be NULL). */
int lc_ct_info(const lc_ct* ct, uint32_t* count, uint32_t* deg, uint32_t* level, double* scale);
/* The handle's device words (evaluation domain), for use with the array calls; NULL for NULL. */
uint64_t* lc_ct_data(const lc_ct* ct);
/* A handle on ciphertexts first .. first+count-1 of `ct`, sharing its memory (the memory lives
 * until the last handle on it is freed).  Views of one handle in order are contiguous, so the
 * evaluation calls use them without copying; other handle sets are gathered first. */
int lc_ct_view(const lc_ct* ct, uint32_t first, uint32_t count, lc_ct** out);
void lc_ct_free(lc_ct* ct);

/* Randomness of key generation, supplied by the caller (host arrays):
 *   pk_a  [n_q][N]  uniform residues (coefficient domain), pk_e [N] errors;
 *   swk_a [1 + n_rot][dnum][n_q + n_p][N], swk_e [1 + n_rot][dnum][N]: the relinearisation key's
 *         first, then one per rotation step in rot_steps order. */
typedef struct {
    const uint64_t* pk_a;
    const int32_t* pk_e;
    const uint64_t* swk_a;
    const int32_t* swk_e;
} lc_keygen_rand;
/* KeyGen (Section "CKKS Scheme Description"; the KGC of Fig. 1): from the ternary secret s
 * (host int8[N]) makes the secret-key handle, the public key ([-a s + e]_Q, a) and the
 * evaluation keys -- the relinearisation key and one rotation key per step in rot_steps[n_rot]
 * (left rotation by that many slots, 1 <= step < N/2, no repeats) -- exactly as lc_pk_gen and
 * lc_evk_add make them.  Any of sk, pk, evk may be NULL to skip it (not all three).
 * Synchronous.  Free with lc_sk_free, lc_pk_free, lc_evk_free. */
int lc_keygen(lc_ctx* ctx, const int8_t* s, const lc_keygen_rand* rand, const int32_t* rot_steps, uint32_t n_rot,
              lc_sk** sk, lc_pk** pk, lc_evk** evk);
void lc_sk_free(lc_sk* sk);
void lc_pk_free(lc_pk* pk);

/* Encryption randomness (host arrays [count][N]): r ternary, e0 and e1 errors. */
typedef struct {
    const int8_t* r;
    const int32_t* e0;
    const int32_t* e1;
} lc_enc_rand;
/* Enc of `count` integer plaintexts m (host int64[count][N]) at level L with the given scale,
 * as lc_encrypt; the new handle has degree 2, level L.  Synchronous. */
int lc_encrypt_plain(lc_ctx* ctx, const lc_pk* pk, const int64_t* m, uint32_t count, double scale,
                     const lc_enc_rand* rand, lc_ct** out);
/* Encode + Enc of real values[len] (host), N/2 slots per ciphertext, the last one zero padded:
 * ceil(len / (N/2)) ciphertexts (rand holds that many rows). */
int lc_encrypt_values(lc_ctx* ctx, const lc_pk* pk, const double* values, size_t len, double scale,
                      const lc_enc_rand* rand, lc_ct** out);
/* Dec + Decode of every ciphertext of a handle with its own level and scale: out[len] (host)
 * receives the N/2 slot values of ciphertext 0, then of ciphertext 1, ... up to len values. */
int lc_decrypt_values(lc_ctx* ctx, const lc_sk* sk, const lc_ct* ct, double* out, size_t len);

/* Encrypted pairwise squared distances (Algorithm 1, "Server Executes") on handles:
 * clients[n], clients[i] holding client i's chunks (count = chunks, the same for every client),
 * each of degree 2 at level L (else LC_ELEVEL) with one common scale (else LC_ESCALE).
 * *out = a new handle of n(n-1)/2 ciphertexts (pairs i<j lexicographic) at level L-1 with scale
 * scale^2 / q_L.  mode, n_groups, groups as in lc_distances. */
int lc_ct_distances(lc_ctx* ctx, const lc_evk* evk, const lc_ct* const* clients, uint32_t n, uint32_t mode,
                    uint32_t n_groups, const uint32_t* groups, lc_ct** out);
/* Masked aggregate (Algorithm 1, "ServerUpdate") on handles: clients as above; masks[n] one
 * ciphertext each at level L with one common scale.  *out = a new handle of `chunks`
 * ciphertexts at level L-1, scale = scale * mask scale / q_L. */
int lc_ct_masked_aggregate(lc_ctx* ctx, const lc_evk* evk, const lc_ct* const* clients, uint32_t n,
                           const lc_ct* const* masks, uint32_t mode, lc_ct** out);

/* One round of one tenant for lc_batch_run: inputs as in lc_ct_distances / lc_ct_masked_aggregate
 * (masks may be NULL: no aggregate; want_dist = 0: no distances), outputs set by the call. */
typedef struct {
    const lc_evk* evk;
    const lc_ct* const* clients;
    uint32_t n;
    const lc_ct* const* masks;
    uint32_t want_dist;
    lc_ct* dist; /* out: n(n-1)/2 distance ciphertexts (NULL if not asked) */
    lc_ct* agg;  /* out: chunks aggregate ciphertexts (NULL without masks) */
} lc_ct_job;
/* Several rounds at once (the uneven multi-job batch): validates every job's handles first
 * (nothing runs if one is malformed), then runs the distances of all jobs through
 * lc_batch_distances and the aggregates through lc_batch_aggregate; flags, n_groups, groups as
 * there.  Each job's results are bit-identical to the same job run alone.  On failure no output
 * handle is left set. */
int lc_batch_run(lc_ctx* ctx, lc_ct_job* jobs, uint32_t n_jobs, uint32_t flags, uint32_t n_groups,
                 const uint32_t* groups);

#ifdef __cplusplus
}
#endif
#endif /* LANCELOT_H */

// Library context: parameters, device tables, scratch and error state.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>
#include <map>
#include <atomic>
#include "../../include/lancelot.h"
#include "modarith.cuh"
#include "ntt.cuh"

#define LC_MAX_SRC 8    // digit size alpha bound
#define LC_MAX_DST 32   // rows of Q_l U P bound
#define LC_MAX_P 8

// ModUp of digit j at level l: y_i = [c_i (D/q_i)^-1]_{q_i} (centred), then for every row t of
// Q_l U P outside the digit: ext_t = sum_i y_i (D/q_i mod m_t) mod m_t.
struct ModUpTab {
    int n_src, n_dst;
    int src_row[LC_MAX_SRC];
    u64 src_q[LC_MAX_SRC];
    u64 hinv[LC_MAX_SRC], hinv_sh[LC_MAX_SRC];
    int dst_row[LC_MAX_DST];
    int dst_mod[LC_MAX_DST];
    u64 hat[LC_MAX_SRC][LC_MAX_DST];   // D/q_i mod m_t
    u64 corr[LC_MAX_SRC][LC_MAX_DST];  // (-q_i * hat) mod m_t, added when y_i is negative
    // reduction constants of each destination modulus m_t (see ModConst)
    u64 dq[LC_MAX_DST], dr64[LC_MAX_DST], dr64sh[LC_MAX_DST], donesh[LC_MAX_DST];
};

// ModDown from Q_l U P to Q_l: y_k = [v_pk (P/p_k)^-1]_{p_k} (centred),
// out_i = (v_i - sum_k y_k (P/p_k mod q_i)) P^-1 mod q_i.
struct ModDownTab {
    int K;
    u64 p[LC_MAX_P];
    u64 phinv[LC_MAX_P], phinv_sh[LC_MAX_P];
    u64 phat[LC_MAX_P][LC_MAX_DST];
    u64 corr[LC_MAX_P][LC_MAX_DST];
    u64 pinv[LC_MAX_DST], pinv_sh[LC_MAX_DST];
    // reduction constants of each q_i (see ModConst)
    u64 qq[LC_MAX_DST], qr64[LC_MAX_DST], qr64sh[LC_MAX_DST], qonesh[LC_MAX_DST];
};

// Rescale at level l: out_i = (x_i - [r]_{q_i}) q_l^-1 for i < l, r the centred last residue.
struct RescaleTab {
    u64 qinv[LC_MAX_DST], qinv_sh[LC_MAX_DST];  // q_l^-1 mod q_i
    u64 negq[LC_MAX_DST];                       // (-q_l) mod q_i
};

// kernel launches issued by this library in this process (all contexts)
extern std::atomic<uint64_t> g_lc_launches;

// per-kernel-class timing (CUDA events on the context stream) for roofline measurement
enum ProfClass { PROF_NTT = 0, PROF_MODUP, PROF_INNER, PROF_MODDOWN, PROF_TENSOR, PROF_RESCALE, PROF_AUTO, PROF_OTHER, PROF_N };
struct ProfRec {
    int cls;
    cudaEvent_t a, b;
    double bytes;
    uint64_t units;
};

struct SwKey {
    u64* data;          // device [dnum][2][n_q+n_p][N], evaluation domain (rotations pre-permuted)
    uint64_t galois;    // 0 for relinearisation
    // rotation keys only: the layout of the one-ModDown group kernel -- not permuted, and rows
    // whose prime is below 2^40 stored as packed 20-bit halves ((v >> 20) << 32 | v mod 2^20)
    u64* qp = nullptr;
};

struct lc_evk {
    lc_ctx* ctx;
    std::map<int32_t, SwKey> keys;  // -1 = relinearisation, r = left rotation by r
};

struct lc_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    lc_allocator alloc{};
    bool has_alloc = false;
    int log_n = 0;
    size_t N = 0;
    int nq = 0, np = 0, dnum = 0, alpha = 0;
    std::vector<u64> mod;  // q_0..q_{nq-1}, p_0..p_{np-1}
    // device tables
    ulonglong2* tw_fwd = nullptr;
    ulonglong2* tw_inv = nullptr;
    ModConst* mc = nullptr;
    ModUpTab* modup = nullptr;        // [nq levels][dnum digits]
    ModDownTab* moddown = nullptr;    // one table (prefixes of Q)
    RescaleTab* rescale = nullptr;    // [nq]
    std::vector<ModConst> mc_host;
    // scratch arena
    void* scratch = nullptr;
    size_t scratch_bytes = 0;
    // staging for host buffers
    void* stage = nullptr;
    size_t stage_bytes = 0;
    // gathered ciphertext handles that are not contiguous (handle calls)
    void* gather = nullptr;
    size_t gather_bytes = 0;
    std::string err;
    uint64_t n_keyswitch = 0, n_modup = 0;
    uint32_t max_batch = 0;  // 0 = limited only by the scratch budget
    // tile-shape choices (LC_TUNE_*, set by lc_set_tuning; results never depend on them)
    int tune[8] = {0, 5, 8, 1, 1, 16, 0, 1};  // [6] LC_TUNE_NTT_ROW_TMA, [7] LC_TUNE_GROUP_KARATSUBA
    bool debug = false;      // LC_DEBUG set: check every launch, remember the first failure
    std::string debug_err;
    bool capturing = false;  // inside lc_graph_begin / lc_graph_end
    uint64_t capture_launches0 = 0;
    // device error word: kernels with bounded waits OR in LC_ERR_* codes; lc_sync reports them
    unsigned* dev_err = nullptr;
    // FP64 encoder (created on first use): slot positions 5^j mod 2N, FFT twiddles, work buffer
    unsigned* enc_pos = nullptr;
    double2* enc_w256 = nullptr;
    double2* enc_wbig = nullptr;
    void* enc_buf = nullptr;
    size_t enc_buf_bytes = 0;
    // overlapped host transfers: one copy stream per direction, one event per ticket
    cudaStream_t copy_stream[2] = {nullptr, nullptr};
    cudaEvent_t compute_mark = nullptr;
    std::vector<cudaEvent_t> copy_events;  // one per ticket slot
    std::vector<uint8_t> copy_busy;         // slot holds a copy not yet waited on
    std::vector<size_t> copy_free;          // reusable slots
    // profiling
    bool prof_on = false;
    std::vector<ProfRec> prof;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;

    NttTables tables() const { return NttTables{tw_fwd, tw_inv, mc, dev_err}; }
    NttTune ntt_tune() const {
        return NttTune{tune[LC_TUNE_NTT_ROW_MINB], tune[LC_TUNE_NTT_COL_MINB], tune[LC_TUNE_NTT_ROW_TMA]};
    }
    int digits(int level) const { return (level + 1 + alpha - 1) / alpha; }
    int qp_mod(int level, int t) const { return t <= level ? t : nq + (t - level - 1); }
};

// allocation through the context's allocator
void* lc_dev_alloc(lc_ctx* c, size_t bytes);
void lc_dev_free(lc_ctx* c, void* p);
// scratch arena of at least `bytes` (grows; contents not preserved across growth)
u64* lc_scratch(lc_ctx* c, size_t bytes);
// status of the launches an entry point just made: the first launch failure recorded in a debug
// context, else cudaGetLastError (LC_OK or LC_ECUDA, message in c->err)
int check_launch(lc_ctx* c, const char* what);
// clears a non-sticky error left on this thread by code outside the library
void clear_prior_error();
// rescale of B ciphertexts using caller-provided scratch `tmp` of rescale_words() words
size_t rescale_words(lc_ctx* c, int B, int deg, int level);
void do_rescale(lc_ctx* c, const u64* ct, int B, int deg, int level, u64* out, u64* tmp);

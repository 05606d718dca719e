// Rescale that allocates nothing: its scratch lives in a fixed device array of this file.
//
// Some callers cannot allocate device memory at the moment they call: a serving process whose
// whole device-memory budget is committed at start-up, code that runs while the caller's
// allocator is locked or must not be re-entered, and latency-sensitive paths that cannot take
// the device-wide synchronisation that cudaMalloc / cudaFree may cause.  For them,
// lc_rescale_noalloc uses this file's static buffer instead of the context's scratch arena,
// which lc_rescale grows on demand.
#include <cuda_runtime.h>
#include <mutex>
#include <string>
#include "context.cuh"

// Maximum scratch of one call: 2 Mi words (16 MiB), enough for one production ciphertext
// (N = 2^15, degree 2, level 14 needs 983,040 words).  Every GPU that loads the library holds
// this array until the process exits.
#define LC_NOALLOC_SCRATCH_WORDS (2u << 20)
static __device__ __align__(256) u64 lc_noalloc_scratch[LC_NOALLOC_SCRATCH_WORDS];

namespace {
std::mutex g_mu;
// Device address of the array, per device ordinal, looked up once.  It stays valid for the
// life of the device's primary context; after cudaDeviceReset (which also invalidates every
// lc_ctx on that device) a process must not call lc_rescale_noalloc on that device again.
u64* g_addr[64] = {nullptr};
}  // namespace

extern "C" int lc_rescale_noalloc(lc_ctx* c, const uint64_t* ct, uint32_t count, uint32_t deg, uint32_t level,
                                  uint64_t* out) {
    if (!c) return LC_EINVAL;
    clear_prior_error();
    if (!ct || !out || level < 1 || (int)level >= c->nq || deg < 1 || deg > 3) {
        c->err = "lc_rescale_noalloc: bad argument";
        return LC_EINVAL;
    }
    if (count == 0) return LC_OK;
    const size_t words = rescale_words(c, (int)count, (int)deg, (int)level);
    if (words > LC_NOALLOC_SCRATCH_WORDS) {
        c->err = "lc_rescale_noalloc: needs " + std::to_string(words * 8) +
                 " bytes of scratch, the static buffer holds " + std::to_string((size_t)LC_NOALLOC_SCRATCH_WORDS * 8) +
                 " (use fewer ciphertexts per call)";
        return LC_EINVAL;
    }
    if (c->device < 0 || c->device >= 64) {
        c->err = "lc_rescale_noalloc: device ordinal out of range";
        return LC_EINVAL;
    }
    u64* scratch = nullptr;
    {
        // one-time set-up per device: the array's device address, looked up with that device current
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_addr[c->device]) {
            int prev = 0;
            if (cudaGetDevice(&prev) != cudaSuccess) {
                cudaGetLastError();
                c->err = "lc_rescale_noalloc: cudaGetDevice failed";
                return LC_ECUDA;
            }
            if (prev != c->device && cudaSetDevice(c->device) != cudaSuccess) {
                cudaGetLastError();
                c->err = "lc_rescale_noalloc: cudaSetDevice failed";
                return LC_ECUDA;
            }
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, lc_noalloc_scratch);
            if (prev != c->device) cudaSetDevice(prev);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                c->err = std::string("lc_rescale_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
                return LC_ECUDA;
            }
            g_addr[c->device] = static_cast<u64*>(p);
        }
        scratch = g_addr[c->device];
    }
    // nothing in the scratch must start at zero: the last-limb copy and the reduced residues are
    // fully written before they are read.  Per-class timing (lc_profile) is skipped for this
    // call: recording it can create CUDA events, and this entry point creates nothing.
    const bool prof = c->prof_on;
    c->prof_on = false;
    do_rescale(c, ct, (int)count, (int)deg, (int)level, out, scratch);
    c->prof_on = prof;
    return check_launch(c, "lc_rescale_noalloc");
}

// Negacyclic NTT / inverse NTT over batches of RNS limbs (the library's "NWT" step).
//
// Domain convention: the forward transform is the Cooley-Tukey network with twiddles
// psi^{br(k)} (br = log2(N)-bit reversal), natural-order input, bit-reversed output:
//   out[idx] = a(psi^(2 br(idx) + 1)) mod q.
// The inverse is the Gentleman-Sande network with psi^{-br(k)}, folded with N^-1.
//
// Layout: every limb is N contiguous words.  The transform is split in two passes so that
// each pass stages a tile in shared memory:
//   column pass  -- stages whose butterfly distance t >= 256 (the top log2(N)-8 index bits);
//                   a CTA owns a 2^C x 16 tile (rows strided by 256 words, 16 columns)
//   row pass     -- stages with t < 256; a CTA owns 8 contiguous blocks of 256 words.
// Inside a pass, each thread runs up to 4 stages (radix 16) in registers between shared
// memory exchanges.  Butterflies are Harvey-lazy: forward values stay in [0, 4q), inverse values in [0, 2q).
#pragma once
#include <cstdint>
#include "modarith.cuh"

#define LC_MAX_ROWS 128

// Which limbs a batched launch touches: limb b (blockIdx.y) is
//   base + (b / n) * batch_stride + row[b % n] * N   with modulus index mod[b % n].
struct RowMap {
    int n;
    uint16_t row[LC_MAX_ROWS];
    uint8_t mod[LC_MAX_ROWS];
};

struct NttTables {
    const ulonglong2* fwd;     // [n_mod][N] {psi^{br(k)}, shoup}
    const ulonglong2* inv;     // [n_mod][N] {psi^{-br(k)}, shoup}; index 0 holds psi^{-br(1)} * N^-1
    const ModConst* mc;        // [n_mod]
    unsigned* err;             // the context's device error word (bounded waits report here)
};

// launch-shape choices (register caps) picked by the tuner; results do not depend on them
struct NttTune {
    int row_minb = 4;  // row pass: minimum resident blocks of 128 threads (4, 5 or 6)
    int col_minb = 8;  // column pass: 1 (no cap), 6, 7 or 8
    int row_tma = 0;   // forward row pass: 1 = persistent blocks streaming tiles with bulk copies
};

void ntt_forward(u64* base, size_t batch_stride, int batch, const RowMap& map, int log_n,
                 const NttTables& t, cudaStream_t s, NttTune tune = NttTune{});
void ntt_inverse(u64* base, size_t batch_stride, int batch, const RowMap& map, int log_n,
                 const NttTables& t, cudaStream_t s, NttTune tune = NttTune{});

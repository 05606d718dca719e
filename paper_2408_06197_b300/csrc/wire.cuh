// Wire form of ciphertext arrays (wire.cu): residues of limb i in w_i bytes, limb after limb.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#define LC_WIRE_MAX_LIMBS 32

struct WireMap {
    int log_n;                          // N = 2^log_n (>= 16)
    int nl;                             // limbs per polynomial
    size_t poly_bytes;                  // bytes of one polynomial (sum of N w_i)
    int w[LC_WIRE_MAX_LIMBS];           // bytes per residue of limb i (4..8)
    size_t off[LC_WIRE_MAX_LIMBS];      // byte offset of limb i inside a polynomial
    uint64_t q[LC_WIRE_MAX_LIMBS];      // the prime of limb i (unpack checks residues < q_i)
};

// polys = count * deg polynomials of m.nl limbs; in/out 16-byte aligned
void wire_unpack(const unsigned char* in, uint64_t* out, size_t polys, const WireMap& m, unsigned* err,
                 cudaStream_t s);
void wire_pack(const uint64_t* in, unsigned char* out, size_t polys, const WireMap& m, cudaStream_t s);

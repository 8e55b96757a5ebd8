// Device-side plan data shared by the kernels.
#pragma once
#include "arith.cuh"

namespace ntt {

// Per-prime constants (one entry per RNS limb prime of a plan).
struct __align__(16) PrimeDev {
    u64 q;
    u64 mu;          // floor(2^{2k} / q), Barrett constant for data x data
    Tw ninv;         // N^{-1} mod q and its Shoup companion
    Tw w1ninv;       // Psi[1] * N^{-1} mod q (the last inverse stage, applied to y - x)
    u32 mbar;        // floor(2^64 / q) (< 2^32 because q > 2^32)
    u32 k;           // bit length of q
};

// Arguments of one pass launch (all limbs of one polynomial batch).
struct PassArgs {
    u64* data;               // [limbs][N], limb-contiguous
    const PrimeDev* primes;  // [L]
    const Tw* tw;            // [L][tw_len] forward table Psi[i] = psi^{brv(i)}
    const Tw* ota;           // [L][2^P] OT A factors for this pass and direction
    const Tw* otb;           // [L][P << s0] OT B factors for this pass and direction
    const u32* prime_map;    // optional [limbs] -> prime index (else limb % L)
    u32 tw_len;              // entries per prime in tw
    u32 n;                   // log2 N
    u32 s0;                  // first stage of the pass
    u32 b;                   // index bits below the pass digit (n - s0 - P)
    u32 L;                   // primes per polynomial
    u32 limb_offset;         // first limb of this launch
};

}  // namespace ntt

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
    u32 rc;          // floor(2^(k+31) / q), the final reduction's reciprocal
    u32 k;           // bit length of q
    u32 rsh;         // k - 28, its shift
};

// Per-prime constants of a 32-bit plan (primes q < 2^28).
struct __align__(16) PrimeDev32 {
    u32 q;
    u32 rc;          // unused by the 32-bit kernels (kept for a common shape)
    Tw32 ninv;       // N^{-1} mod q and its Shoup companion
    Tw32 w1ninv;     // Psi[1] * N^{-1} mod q (the last inverse stage, applied to y - x)
    u32 k;           // bit length of q
    u32 rsh;         // unused by the 32-bit kernels
};

// Word-size traits of the pass kernels: the data word, the twiddle pair and
// the per-prime constants.
template <class W>
struct WordTypes;
template <>
struct WordTypes<u64> {
    using Tw = ntt::Tw;
    using Prime = PrimeDev;
};
template <>
struct WordTypes<u32> {
    using Tw = Tw32;
    using Prime = PrimeDev32;
};

// Arguments of one pass launch (all limbs of one polynomial batch).
template <class W = u64>
struct PassArgsT {
    using TwT = typename WordTypes<W>::Tw;
    using PrimeT = typename WordTypes<W>::Prime;
    W* data;                 // [limbs][N], limb-contiguous
    const PrimeT* primes;    // [L]
    const TwT* tw;           // [L][tw_len] forward table Psi[i] = psi^{brv(i)}
    const TwT* ota;          // [L][2^P] OT A factors for this pass and direction
    const TwT* otb;          // [L][P << s0] OT B factors for this pass and direction
    const u32* prime_map;    // optional [limbs] -> prime index (else limb % L)
    u32 tw_len;              // entries per prime in tw
    u32 n;                   // log2 N
    u32 s0;                  // first stage of the pass
    u32 b;                   // index bits below the pass digit (n - s0 - P)
    u32 L;                   // primes per polynomial
    u32 limb_offset;         // first limb of this launch
};
using PassArgs = PassArgsT<u64>;

}  // namespace ntt

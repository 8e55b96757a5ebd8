// Modular arithmetic for the NTT kernels (device side).
//
// Word size 64 bit, primes 2^32 < q < 2^60 (the paper uses 2^59 < p < 2^60,
// Sec. IV "32b vs. 64b word size").  Because q < 2^60, any value below 16q
// fits in a word, so the butterflies keep values lazily in [0, X*q) for a
// compile-time bound X <= 16 and reduce only when the bound would overflow.
//
// shoup_lazy is Shoup's modular multiplication (Algorithm 4) with the
// quotient estimated from three 32x32-bit partial products instead of the
// exact high word of the 128-bit product (w' = floor(w 2^64 / q)):
//   qhat = yh*wh' + hi32(yh*wl') + hi32(yl*wh')
//   r    = lo64(y*w + qhat*(2^64 - q))  =  y*w - qhat*q  mod 2^64
// For every y < 2^64 and w < q the exact quotient floor(y w / q) exceeds qhat
// by at most 3, so r lies in [0, 4q).  (Dropped: lo32 parts of both middle
// products and the low product, each < 1 in units of 2^64, and < 1 from the
// floor in w'.)  The products are written as PTX 32-bit multiplies so that
// each maps to one multiply-pipe instruction: two high products and one wide
// multiply-add (their sum as its addend) for qhat, two wide and four low
// products for r.
#pragma once
#include <stdint.h>

namespace ntt {

typedef unsigned long long u64;
typedef unsigned int u32;

struct __align__(16) Tw {      // a twiddle and its Shoup companion
    u64 w, wp;
};

__device__ __forceinline__ u32 lo32(u64 x) { return (u32)x; }
__device__ __forceinline__ u32 hi32(u64 x) { return (u32)(x >> 32); }

__device__ __forceinline__ u64 mul_wide(u32 a, u32 b) { return (u64)a * (u64)b; }

// y * w mod q, result in [0, 4q), any 64-bit y.
__device__ __forceinline__ u64 shoup_lazy(u64 y, u64 w, u64 wp, u64 q)
{
    const u32 yl = lo32(y), yh = hi32(y);
    const u64 nq = 0ull - q;      // 2^64 - q
    u64 r;
    u32 h1, h2;
    asm("mul.hi.u32 %0, %1, %2;" : "=r"(h1) : "r"(yh), "r"(lo32(wp)));
    asm("mul.hi.u32 %0, %1, %2;" : "=r"(h2) : "r"(yl), "r"(hi32(wp)));
    u64 qhat;   // yh*wh' + h1 + h2: the two high parts as the wide product's addend
    asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(qhat) : "r"(yh), "r"(hi32(wp)), "l"((u64)h1 + h2));
    // low word of y*w + qhat*nq: the low partial products in 64 bits (a carry
    // out of bit 63 is a multiple of 2^64 and drops out), then the four
    // cross products into the high word
    asm("mul.wide.u32 %0, %1, %2;" : "=l"(r) : "r"(yl), "r"(lo32(w)));
    asm("mad.wide.u32 %0, %1, %2, %0;" : "+l"(r) : "r"(lo32(qhat)), "r"(lo32(nq)));
    u32 rh = hi32(r);
    asm("mad.lo.u32 %0, %1, %2, %0;" : "+r"(rh) : "r"(yl), "r"(hi32(w)));
    asm("mad.lo.u32 %0, %1, %2, %0;" : "+r"(rh) : "r"(yh), "r"(lo32(w)));
    asm("mad.lo.u32 %0, %1, %2, %0;" : "+r"(rh) : "r"(lo32(qhat)), "r"(hi32(nq)));
    asm("mad.lo.u32 %0, %1, %2, %0;" : "+r"(rh) : "r"(hi32(qhat)), "r"(lo32(nq)));
    return ((u64)rh << 32) | lo32(r);
}

// x in [0, 2c) -> [0, c), for c <= 2^63: x - c wraps to at least 2^63 exactly
// when x < c, so its sign bit decides (one test of the high word).
__device__ __forceinline__ u64 csub(u64 x, u64 c)
{
    const u64 d = x - c;
    return (long long)d < 0 ? x : d;
}

// x mod q into [0, 2q) for x < 16 q.  k is the bit length of q, sh = k - 28,
// rc = floor(2^(k+31) / q) (2^31 <= rc < 2^32).  The quotient estimate
//   kq = floor(floor(x / 2^sh) rc / 2^59)
// uses the top 32 bits of x (x < 2^(k+4)).  Dropping the low sh bits of x
// loses under 2^sh / q < 2^-27 of a quotient unit and truncating rc under
// 2^32 / 2^59, so kq is floor(x / q) or one less.
__device__ __forceinline__ u64 reduce2(u64 x, u64 q, u32 rc, u32 sh)
{
    u32 xs;
    asm("shf.r.clamp.b32 %0, %1, %2, %3;" : "=r"(xs) : "r"(lo32(x)), "r"(hi32(x)), "r"(sh));
    const u32 kq = hi32(mul_wide(xs, rc)) >> 27;
    return x - (u64)kq * q;
}

// Bring x in [0, X q) to [0, q), X a compile-time bound <= 16.
template <int X>
__device__ __forceinline__ u64 canon(u64 x, u64 q, u32 rc, u32 sh)
{
    static_assert(X >= 1 && X <= 16, "range");
    if (X > 4) return csub(reduce2(x, q, rc, sh), q);
    if (X > 2) x = csub(x, 2 * q);
    if (X > 1) x = csub(x, q);
    return x;
}

// ---------------------------------------------------------------------------
// Range bookkeeping for the forward (Cooley-Tukey) butterfly
//   x' = x + t,  y' = x + 4q - t,   t = shoup_lazy(y, w) in [0, 4q)
// Inputs of a stage lie in [0, X q); outputs in [0, (X + 4) q).  When X + 4
// would exceed 16, the x operand is first brought below 8q by one
// conditional subtraction of 8q (integer ALU work, which leaves the multiply
// pipe to the Shoup products), so the outputs lie in [0, 12q).  From a
// canonical input the bounds run 1, 5, 9, 13, 12, 16, 12, 16, ...
// ---------------------------------------------------------------------------
__host__ __device__ constexpr bool ct_reduces(int X) { return X + 4 > 16; }
__host__ __device__ constexpr int ct_next(int X) { return ct_reduces(X) ? 12 : X + 4; }
__host__ __device__ constexpr int ct_range_after(int X, int stages)
{
    return stages == 0 ? X : ct_range_after(ct_next(X), stages - 1);
}

template <int X>
__device__ __forceinline__ void ct_bfly(u64& x, u64& y, const u64 w, const u64 wp,
                                        const u64 q, const u64 q4)
{
    u64 a = x;
    if (ct_reduces(X)) a = csub(a, q4 << 1);
    const u64 t = shoup_lazy(y, w, wp, q);
    x = a + t;
    y = a + q4 - t;
}

// same, with the twiddle applied as two factors (on-the-fly twiddling):
// t = (y * w1) * w2, each a Shoup product
template <int X>
__device__ __forceinline__ void ct_bfly_ot(u64& x, u64& y, const Tw f1, const Tw f2,
                                           const u64 q, const u64 q4)
{
    u64 a = x;
    if (ct_reduces(X)) a = csub(a, q4 << 1);
    const u64 t = shoup_lazy(shoup_lazy(y, f1.w, f1.wp, q), f2.w, f2.wp, q);
    x = a + t;
    y = a + q4 - t;
}

// ---------------------------------------------------------------------------
// Range bookkeeping for the inverse (Gentleman-Sande) butterfly
//   x' = x + y,  y' = shoup_lazy(d, w)  with d = x - y + X q  (or y - x + X q
//   when the twiddle is stored negated).
// Inputs in [0, X q) need X <= 8 (x + y < 16 q).  y' is in [0, 4q); x' in
// [0, 2X q) and, when 2X > 8, is brought below 8q by one conditional
// subtraction of 8q, so the next stage again sees X <= 8.  From a canonical
// input the bounds run 1, 4, 8, 8, 8, ...
// ---------------------------------------------------------------------------
__host__ __device__ constexpr bool gs_reduces(int X) { return 2 * X > 8; }
__host__ __device__ constexpr int gs_next(int X)
{
    return gs_reduces(X) ? 8 : (2 * X > 4 ? 2 * X : 4);
}
__host__ __device__ constexpr int gs_range_after(int X, int stages)
{
    return stages == 0 ? X : gs_range_after(gs_next(X), stages - 1);
}

// Bound of one slot in a round of GS stages held in registers, smallest
// stride first.  The round's stage b pairs the slots that differ in bit b of
// the slot index, so after stages 0 .. b-1 a slot's bound depends only on its
// bits below b: a 1 made it a product output (below 4q), a 0 a sum (twice the
// bound, brought back below 8q when that would pass 8q).  The two slots of a
// pair therefore share the bound gs_slot_bound(X, b, i) (i: the bits below b,
// X: the round's input bound), and only a sum of two values that may exceed 4q
// needs the subtraction: 20 of the 32 that the uniform bound gs_next spends
// on a radix-16 round from 8q.  Never above gs_range_after(X, b).
__host__ __device__ constexpr int gs_slot_bound(int X, int b, int i)
{
    for (int j = 0; j < b; ++j) X = ((i >> j) & 1) ? 4 : (gs_reduces(X) ? 8 : 2 * X);
    return X;
}
__host__ __device__ constexpr bool gs_slot_bounds_hold()
{
    for (int X = 1; X <= 8; ++X)
        for (int b = 0; b <= 6; ++b)
            for (int i = 0; i < (1 << b); ++i)
                if (gs_slot_bound(X, b, i) > 8 || gs_slot_bound(X, b, i) > gs_range_after(X, b)) return false;
    return true;
}
static_assert(gs_slot_bounds_hold(), "per-slot GS bounds within the uniform ones");

// NEG: twiddle stored as -w (the forward table read backwards), so the
// difference is taken as y - x.
template <int X, bool NEG>
__device__ __forceinline__ void gs_bfly(u64& x, u64& y, const u64 w, const u64 wp,
                                        const u64 q)
{
    static_assert(X <= 8, "GS inputs must stay below 8q");
    const u64 Xq = (u64)X * q;
    const u64 d = NEG ? (y + Xq - x) : (x + Xq - y);
    u64 s = x + y;
    if (gs_reduces(X)) s = csub(s, q << 3);
    x = s;
    y = shoup_lazy(d, w, wp, q);
}

template <int X, bool NEG>
__device__ __forceinline__ void gs_bfly_ot(u64& x, u64& y, const Tw f1, const Tw f2,
                                           const u64 q)
{
    static_assert(X <= 8, "GS inputs must stay below 8q");
    const u64 Xq = (u64)X * q;
    const u64 d = NEG ? (y + Xq - x) : (x + Xq - y);
    u64 s = x + y;
    if (gs_reduces(X)) s = csub(s, q << 3);
    x = s;
    y = shoup_lazy(shoup_lazy(d, f1.w, f1.wp, q), f2.w, f2.wp, q);
}

// Last inverse stage with N^{-1} folded in:
//   x' = (x + y) N^{-1},  y' = d * (w N^{-1});  both in [0, 4q).
template <int X, bool NEG>
__device__ __forceinline__ void gs_bfly_scaled(u64& x, u64& y, const Tw wn, const Tw ninv,
                                               const u64 q)
{
    static_assert(X <= 8, "GS inputs must stay below 8q");
    const u64 Xq = (u64)X * q;
    const u64 d = NEG ? (y + Xq - x) : (x + Xq - y);
    x = shoup_lazy(x + y, ninv.w, ninv.wp, q);
    y = shoup_lazy(d, wn.w, wn.wp, q);
}

// ---------------------------------------------------------------------------
// 32-bit words.  Primes q < 2^28, so every value below 16q fits a word and the
// range bookkeeping above applies unchanged.  Shoup's product takes the exact
// quotient estimate qhat = hi32(y w'), w' = floor(w 2^32 / q): for y < 2^32,
// floor(y w / q) - qhat <= 1, so r = lo32(y w - qhat q) lies in [0, 2q), within
// the [0, 4q) the butterflies allow.
// ---------------------------------------------------------------------------
struct __align__(8) Tw32 {     // a twiddle and its 32-bit Shoup companion
    u32 w, wp;
};

__device__ __forceinline__ u32 shoup_lazy(u32 y, u32 w, u32 wp, u32 q)
{
    const u32 qhat = __umulhi(y, wp);
    return y * w - qhat * q;      // exact value < 2q
}

// x in [0, 2c) -> [0, c): x - c wraps above x exactly when x < c
__device__ __forceinline__ u32 csub(u32 x, u32 c) { return min(x, x - c); }

template <int X>
__device__ __forceinline__ u32 canon(u32 x, u32 q, u32, u32)
{
    static_assert(X >= 1 && X <= 16, "range");
    if (X > 8) x = csub(x, q << 3);
    if (X > 4) x = csub(x, q << 2);
    if (X > 2) x = csub(x, q << 1);
    if (X > 1) x = csub(x, q);
    return x;
}

template <int X>
__device__ __forceinline__ void ct_bfly(u32& x, u32& y, const u32 w, const u32 wp, const u32 q, const u32 q4)
{
    u32 a = x;
    if (ct_reduces(X)) a = csub(a, q4 << 1);
    const u32 t = shoup_lazy(y, w, wp, q);
    x = a + t;
    y = a + q4 - t;
}

template <int X>
__device__ __forceinline__ void ct_bfly_ot(u32& x, u32& y, const Tw32 f1, const Tw32 f2, const u32 q,
                                           const u32 q4)
{
    u32 a = x;
    if (ct_reduces(X)) a = csub(a, q4 << 1);
    const u32 t = shoup_lazy(shoup_lazy(y, f1.w, f1.wp, q), f2.w, f2.wp, q);
    x = a + t;
    y = a + q4 - t;
}

template <int X, bool NEG>
__device__ __forceinline__ void gs_bfly(u32& x, u32& y, const u32 w, const u32 wp, const u32 q)
{
    static_assert(X <= 8, "GS inputs must stay below 8q");
    const u32 Xq = (u32)X * q;
    const u32 d = NEG ? (y + Xq - x) : (x + Xq - y);
    u32 s = x + y;
    if (gs_reduces(X)) s = csub(s, q << 3);
    x = s;
    y = shoup_lazy(d, w, wp, q);
}

template <int X, bool NEG>
__device__ __forceinline__ void gs_bfly_ot(u32& x, u32& y, const Tw32 f1, const Tw32 f2, const u32 q)
{
    static_assert(X <= 8, "GS inputs must stay below 8q");
    const u32 Xq = (u32)X * q;
    const u32 d = NEG ? (y + Xq - x) : (x + Xq - y);
    u32 s = x + y;
    if (gs_reduces(X)) s = csub(s, q << 3);
    x = s;
    y = shoup_lazy(shoup_lazy(d, f1.w, f1.wp, q), f2.w, f2.wp, q);
}

template <int X, bool NEG>
__device__ __forceinline__ void gs_bfly_scaled(u32& x, u32& y, const Tw32 wn, const Tw32 ninv, const u32 q)
{
    static_assert(X <= 8, "GS inputs must stay below 8q");
    const u32 Xq = (u32)X * q;
    const u32 d = NEG ? (y + Xq - x) : (x + Xq - y);
    x = shoup_lazy(x + y, ninv.w, ninv.wp, q);
    y = shoup_lazy(d, wn.w, wn.wp, q);
}

// Barrett product of two residues a, b < q (data times data, no companion;
// Barrett, CRYPTO 1986).  k = bit length of q, mu = floor(2^{2k} / q) < 2^{k+1}:
//   t = floor(ab / 2^{k-1}),  qhat = floor(t mu / 2^{k+1}),  r = ab - qhat q
// and qhat is at most 2 below floor(ab / q), so r lies in [0, 3q).
__device__ __forceinline__ u64 mulmod_barrett(u64 a, u64 b, u64 q, u64 mu, u32 k)
{
    const u64 lo = a * b, hi = __umul64hi(a, b);
    const u64 t = (hi << (65 - k)) | (lo >> (k - 1));   // k in [33, 60]
    const u64 plo = t * mu, phi = __umul64hi(t, mu);
    const u64 qhat = (phi << (63 - k)) | (plo >> (k + 1));
    return lo - qhat * q;
}

}  // namespace ntt

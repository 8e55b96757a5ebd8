// One pass of the negacyclic NTT over a tile of sub-transforms.
//
// The forward transform is Algorithm 1 (Cooley-Tukey, natural order in,
// bit-reversed order out, Psi[i] = psi^{brv(i)}): stage s (0 <= s < n) pairs
// indices that differ in bit n-1-s, with twiddle Psi[2^s + (index >> (n-s))].
// The inverse is the Gentleman-Sande network that undoes it stage by stage
// (Sec. III-A: the Psi^{-1} twist is merged into the iNTT), followed by the
// N^{-1} scaling, which is folded into the last stage.
//
// A pass covers P consecutive stages [s0, s0 + P).  Those stages only mix
// indices that agree outside bits [b, b + P), b = n - s0 - P, so the pass is
// a set of N / 2^P independent 2^P-point sub-transforms ("SMEM implementation"
// of Sec. VI-C, Kernel-1 / Kernel-2 when there are two passes).  A CTA loads a
// tile of C = 2^LOGC sub-transforms into shared memory, runs the P stages in
// rounds of at most KMAX stages per thread held in registers (the per-thread
// NTT of Sec. VI-C), and writes the tile back.
//   ROWS  : b == 0, the tile is C consecutive rows of 2^P contiguous words.
//   !ROWS : b >= LOGC, the tile is 2^P rows (stride 2^b) of C contiguous words
//           (the coalesced Kernel-1 of Sec. VI-C: adjacent sub-transforms per
//           CTA so that every row segment is a full line).
// Values stay lazy between stages and passes (see arith.cuh); the final pass
// writes canonical residues.
#pragma once
#include "arith.cuh"
#include "device_types.cuh"

namespace ntt {

__host__ __device__ constexpr int nrounds(int P, int KMAX) { return (P + KMAX - 1) / KMAX; }
__host__ __device__ constexpr int rsize(int P, int KMAX, int r)
{
    return P / nrounds(P, KMAX) + (r < P % nrounds(P, KMAX) ? 1 : 0);
}
__host__ __device__ constexpr int rstart(int P, int KMAX, int r)
{
    return r == 0 ? 0 : rstart(P, KMAX, r - 1) + rsize(P, KMAX, r - 1);
}
__host__ __device__ constexpr int pass_threads(int P, int LOGC, int KMAX)
{
    return 1 << (LOGC + P - rsize(P, KMAX, 0));
}
__host__ __device__ constexpr int ct_range_max(int X, int stages)
{
    return stages == 0 ? X : (X > ct_range_max(ct_next(X), stages - 1) ? X : ct_range_max(ct_next(X), stages - 1));
}
__host__ __device__ constexpr int gs_range_max(int X, int stages)
{
    return stages == 0 ? X : (X > gs_range_max(gs_next(X), stages - 1) ? X : gs_range_max(gs_next(X), stages - 1));
}

// Shared-memory word swizzle: 16-byte chunk index XOR (line index mod 8),
// line = 16 words.  Keeps word pairs together (16-byte accesses) and makes the
// strided per-thread accesses of every round conflict-free.
__device__ __forceinline__ u32 swz(u32 w) { return w ^ (((w >> 4) & 7u) << 1); }

// The same for 32-bit words: 16-byte chunk index XOR (line index mod 8), line
// = 32 words (128 bytes), which is the TMA 128-byte swizzle for 4-byte
// elements; quads, hence word pairs, stay together.
template <class W>
__device__ __forceinline__ u32 swzw(u32 w)
{
    if constexpr (sizeof(W) == 8) return swz(w);
    else return w ^ (((w >> 5) & 7u) << 2);
}

// Twiddle slots.  Within stage s the butterfly with index j = (u << sl) |
// (hi << k) | pre (u: sub-transform bits, hi: bits of the round digit fixed
// per thread, pre: the butterfly's group inside the thread's radix-2^KR
// block, k = sl - K0) reads table slot (u << sl) | (pre << K0) | hi, so that
// for each pre the lanes of a warp (consecutive hi) read consecutive slots.
// The plan stores Psi in that order (tw_slot); the order is a bit
// permutation, so complementing j complements its slot and the inverse can
// still read Psi^{-1}[2^s + j] = -Psi[2^{s+1} - 1 - j] at the mirrored slot.
__host__ __device__ constexpr unsigned tw_slot(unsigned j, int sl, int K0, int k)
{
    return (j >> sl << sl) | ((j & ((1u << k) - 1u)) << K0) | ((j >> k) & ((1u << K0) - 1u));
}

// Everything one item (one thread's 2^KR elements of one sub-transform in one
// round) needs besides its data.
template <class W = u64>
struct ItemCtxT {
    using TwT = typename WordTypes<W>::Tw;
    const TwT* tw;       // twiddle table base for this prime (smem or global)
    const TwT* ota;      // OT A factors for this prime (smem)
    const TwT* otb;      // OT B factors for this prime (global)
    W q, q4;
    u32 rc, rsh;         // final reduction constants
    u32 u;               // upper index bits (which 2^{n-s0} block)
    u32 ubase;           // first block of the tile (staged twiddle runs are per tile)
    u32 hi;              // bits of v above the round digit
    u32 s0;              // first stage of the pass
    TwT ninv, w1ninv;
    const TwT* twg;      // the prime's full table in global memory (SOT 2: the last stage's twiddles)
};
using ItemCtx = ItemCtxT<u64>;

// two consecutive words as one vector (16 bytes for 64-bit words, 8 for 32-bit)
__device__ __forceinline__ void load_pair(const u64* p, u64& a, u64& b)
{
    const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(p);
    a = v.x;
    b = v.y;
}
__device__ __forceinline__ void load_pair(const u32* p, u32& a, u32& b)
{
    const uint2 v = *reinterpret_cast<const uint2*>(p);
    a = v.x;
    b = v.y;
}
__device__ __forceinline__ void store_pair(u64* p, u64 a, u64 b)
{
    *reinterpret_cast<ulonglong2*>(p) = make_ulonglong2(a, b);
}
__device__ __forceinline__ void store_pair(u32* p, u32 a, u32 b) { *reinterpret_cast<uint2*>(p) = make_uint2(a, b); }
template <class W>
struct PairVec;
template <>
struct PairVec<u64> {
    using T = ulonglong2;
};
template <>
struct PairVec<u32> {
    using T = uint2;
};

// ------------------------------------------------------- twiddle sources --
// Where a round reads the table twiddle of stage sl (of the pass), slot jlo:
//   TW_PASS   : the pass's own table Psi[0, 2^P) in shared memory (a pass that
//               holds stage 0, where that is all it needs);
//   TW_GLOBAL : the prime's full table in global memory;
//   TW_STAGED : runs of the full table copied into shared memory for the
//               tile's SCR consecutive blocks u0 .. u0 + SCR - 1: stage sl's
//               run holds entries [2^(s0+sl) + (u0 << sl), + (SCR << sl)) (the
//               forward) or the mirrored run the inverse reads, at offset
//               SCR (2^sl - 2^SSB) of the buffer (SSB: its first stage).
// The inverse reads Psi^{-1}[2^s + j] = -Psi[2^{s+1} - 1 - j].
enum : int { TW_PASS = 0, TW_GLOBAL = 1, TW_STAGED = 2 };

template <int TWM, int SCR, int SSB, int sl, bool FWDDIR, class W>
__device__ __forceinline__ u32 tw_index(const ItemCtxT<W>& c, const u32 jlo)
{
    if constexpr (TWM == TW_PASS) {
        return FWDDIR ? (1u << sl) + jlo : (2u << sl) - 1u - jlo;
    } else if constexpr (TWM == TW_GLOBAL) {
        const u32 j = (c.u << sl) + jlo;
        return FWDDIR ? (1u << (c.s0 + sl)) + j : (2u << (c.s0 + sl)) - 1u - j;
    } else {
        static_assert(sl >= SSB, "stage below the buffer's first stage");
        constexpr u32 off = (u32)SCR * ((1u << sl) - (1u << SSB));
        const u32 r = c.u - c.ubase;
        return FWDDIR ? off + (r << sl) + jlo : off + (((u32)SCR - r) << sl) - 1u - jlo;
    }
}

// OT factors of stage sl (one of the last OTS stages): the per-row factor
// B[sl][u] and the per-position factor A[2^sl + j].  SOT: both are staged in
// shared memory with the tile (A from entry 2^(P-OTS), B as OTS runs of SCR
// rows), else read from the prime's global tables.  SOT 2 (a table-mode row
// pass with the OT staging layout and OTS 1): the last stage is not
// factored; its plain table twiddles come from the table in global memory
// (`twg`), loaded into registers at the start of the round that holds it.
template <int P, int OTS, int SOT, int SCR, int sl, class W>
__device__ __forceinline__ void ot_factors(const ItemCtxT<W>& c, const u32 jlo, typename WordTypes<W>::Tw& f1,
                                           typename WordTypes<W>::Tw& f2)
{
    if constexpr (SOT) {
        f1 = c.otb[(u32)(sl - (P - OTS)) * SCR + (c.u - c.ubase)];
        f2 = c.ota[(1u << sl) + jlo - (1u << (P - OTS))];
    } else {
        f1 = c.otb[((u32)sl << c.s0) + c.u];
        f2 = c.ota[(1u << sl) + jlo];
    }
}

// ---------------------------------------------------------------- forward --
template <int P, int KR, int K0, int k, int X, int OTS, int TWM, int SCR, int SSB, int SOT, int E, class W>
__device__ __forceinline__ void fwd_stages(W (&x)[E], const ItemCtxT<W>& c,
                                           const typename WordTypes<W>::Tw (&t0)[(E >> 1) > 0 ? (E >> 1) : 1])
{
    if constexpr (k < KR) {
        constexpr int half = E >> (k + 1);
        constexpr int sl = K0 + k;                  // stage within the pass
        constexpr bool ot = sl >= P - OTS;
#pragma unroll
        for (int pre = 0; pre < (1 << k); ++pre) {
            const u32 jlo = ((u32)pre << K0) | c.hi;      // twiddle slot, see tw_slot
            if constexpr (ot && SOT == 2) {
                const auto t = k == KR - 1 ? t0[pre] : c.twg[tw_index<TW_GLOBAL, SCR, SSB, sl, true>(c, jlo)];
#pragma unroll
                for (int i = 0; i < half; ++i)
                    ct_bfly<X>(x[pre * 2 * half + i], x[pre * 2 * half + i + half], t.w, t.wp, c.q, c.q4);
            } else if constexpr (ot) {
                typename WordTypes<W>::Tw f1, f2;
                ot_factors<P, OTS, SOT, SCR, sl>(c, jlo, f1, f2);
#pragma unroll
                for (int i = 0; i < half; ++i)
                    ct_bfly_ot<X>(x[pre * 2 * half + i], x[pre * 2 * half + i + half], f1, f2, c.q, c.q4);
            } else {
                const auto t = c.tw[tw_index<TWM, SCR, SSB, sl, true>(c, jlo)];
#pragma unroll
                for (int i = 0; i < half; ++i)
                    ct_bfly<X>(x[pre * 2 * half + i], x[pre * 2 * half + i + half], t.w, t.wp, c.q, c.q4);
            }
        }
        fwd_stages<P, KR, K0, k + 1, ct_next(X), OTS, TWM, SCR, SSB, SOT, E>(x, c, t0);
    }
}

// Compile-time loop: f(SlotIdx<I>{}) for I = I0 .. N-1.
template <int I>
struct SlotIdx {
    static constexpr int value = I;
};
template <int I, int N, class F>
__device__ __forceinline__ void static_for(F&& f)
{
    if constexpr (I < N) {
        f(SlotIdx<I>{});
        static_for<I + 1, N>(f);
    }
}

// ---------------------------------------------------------------- inverse --
// Whether the first stage an inverse round runs (its largest, 2^{KR-1}
// twiddles per item) reads table twiddles from global memory; those are then
// loaded before the round's shared-memory reads, to overlap their latency.
template <int P, int KR, int K0, int OTS, bool HAS_S0, int TWM>
__host__ __device__ constexpr bool inv_preloads()
{
    return TWM == TW_GLOBAL && K0 + KR - 1 < P - OTS && !(HAS_S0 && K0 == 0 && KR == 1);
}

// Stages run from KR-1 down to 0.  HAS_S0: this round holds global stage 0
// (K0 == 0 and s0 == 0), whose butterfly also applies N^{-1}.  t0: the
// twiddles of stage KR-1 when inv_preloads().
template <int P, int KR, int K0, int k, int X, int OTS, bool HAS_S0, int TWM, int SCR, int SSB, int SOT, bool PRE,
          int E, class W>
__device__ __forceinline__ void inv_stages(W (&x)[E], const ItemCtxT<W>& c,
                                           const typename WordTypes<W>::Tw (&t0)[(E >> 1) > 0 ? (E >> 1) : 1])
{
    if constexpr (k >= 0) {
        constexpr int half = E >> (k + 1);
        constexpr int b = KR - 1 - k;               // this stage pairs slots differing in bit b
        constexpr int sl = K0 + k;
        constexpr bool ot = sl >= P - OTS;
        static_assert(X <= 8, "GS inputs must stay below 8q");
        if constexpr (HAS_S0 && K0 == 0 && k == 0) {
            // global stage 0: a single twiddle Psi^{-1}[1] = -Psi[1]
            static_for<0, half>([&](auto I) {
                constexpr int XS = gs_slot_bound(X, b, decltype(I)::value);
                gs_bfly_scaled<XS, true>(x[I.value], x[I.value + half], c.w1ninv, c.ninv, c.q);
            });
        } else {
#pragma unroll
            for (int pre = 0; pre < (1 << k); ++pre) {
                const u32 jlo = ((u32)pre << K0) | c.hi;  // twiddle slot, see tw_slot
                const int base = pre * 2 * half;
                if constexpr (ot && SOT == 2) {
                    const auto t = k == KR - 1 ? t0[pre] : c.twg[tw_index<TW_GLOBAL, SCR, SSB, sl, false>(c, jlo)];
                    static_for<0, half>([&](auto I) {
                        constexpr int XS = gs_slot_bound(X, b, decltype(I)::value);
                        gs_bfly<XS, true>(x[base + I.value], x[base + I.value + half], t.w, t.wp, c.q);
                    });
                } else if constexpr (ot) {
                    typename WordTypes<W>::Tw f1, f2;
                    ot_factors<P, OTS, SOT, SCR, sl>(c, jlo, f1, f2);
                    static_for<0, half>([&](auto I) {
                        constexpr int XS = gs_slot_bound(X, b, decltype(I)::value);
                        gs_bfly_ot<XS, false>(x[base + I.value], x[base + I.value + half], f1, f2, c.q);
                    });
                } else {
                    constexpr bool pre_loaded = PRE && k == KR - 1 && inv_preloads<P, KR, K0, OTS, HAS_S0, TWM>();
                    const auto t = pre_loaded ? t0[pre] : c.tw[tw_index<TWM, SCR, SSB, sl, false>(c, jlo)];
                    static_for<0, half>([&](auto I) {
                        constexpr int XS = gs_slot_bound(X, b, decltype(I)::value);
                        gs_bfly<XS, true>(x[base + I.value], x[base + I.value + half], t.w, t.wp, c.q);
                    });
                }
            }
        }
        // X stays the round's input bound: each slot's bound follows from it
        inv_stages<P, KR, K0, k - 1, X, OTS, HAS_S0, TWM, SCR, SSB, SOT, PRE, E>(x, c, t0);
    }
}

// ------------------------------------------------------------------ round --
// One round: every item of the tile reads its 2^KR elements from shared
// memory, runs KR stages in registers and writes them back.
// PRE: an inverse round loads the global twiddles of its first stage before
// its shared-memory reads (see inv_preloads).
template <int P, int LOGC, int KMAX, int r, bool ROWS, bool FWD, int XR, int OTS, bool HAS_S0, int CANON, int TWM,
          int SCR, int SSB, int SOT, int NT, bool PRE, class W>
__device__ __forceinline__ void run_round(W* sm, ItemCtxT<W> c, const u32 u_base, const u32 tid)
{
    constexpr int KR = rsize(P, KMAX, r);
    constexpr int K0 = rstart(P, KMAX, r);
    constexpr int E = 1 << KR;
    constexpr int NLO = P - K0 - KR;              // bits of v below the digit
    constexpr int R = 1 << P, C = 1 << LOGC;
    constexpr int ITEMS = C << (P - KR);
    constexpr bool PAIRS = ROWS && NLO == 0 && E >= 2;   // contiguous in smem
#pragma unroll 1
    for (int it = tid; it < ITEMS; it += NT) {
        u32 cc, hi, lo;
        if constexpr (ROWS) {
            lo = (u32)it & ((1u << NLO) - 1u);
            hi = ((u32)it >> NLO) & ((1u << K0) - 1u);
            cc = (u32)it >> (NLO + K0);
        } else {
            cc = (u32)it & (C - 1u);
            lo = ((u32)it >> LOGC) & ((1u << NLO) - 1u);
            hi = (u32)it >> (LOGC + NLO);
        }
        c.hi = hi;
        if constexpr (ROWS) c.u = u_base + cc;
        const u32 vbase = (hi << (P - K0)) | lo;
        typename WordTypes<W>::Tw t0[(E >> 1) > 0 ? (E >> 1) : 1];
        if constexpr (!FWD && PRE && inv_preloads<P, KR, K0, OTS, HAS_S0, TWM>()) {
#pragma unroll
            for (int pre = 0; pre < (E >> 1); ++pre)
                t0[pre] = c.tw[tw_index<TWM, SCR, SSB, K0 + KR - 1, false>(c, ((u32)pre << K0) | hi)];
        }
        if constexpr (SOT == 2 && K0 + KR - 1 >= P - OTS) {
            // the last stage's table twiddles come from global memory: load
            // them before the round's shared-memory reads (t0 serves the
            // round's last forward stage or its first inverse stage)
#pragma unroll
            for (int pre = 0; pre < (E >> 1); ++pre)
                t0[pre] = c.twg[tw_index<TW_GLOBAL, SCR, SSB, K0 + KR - 1, FWD>(c, ((u32)pre << K0) | hi)];
        }
        W x[E];
        if constexpr (PAIRS) {
#pragma unroll
            for (int i = 0; i < E; i += 2) {
                const u32 w = cc * R + vbase + (u32)i;
                load_pair(sm + swzw<W>(w), x[i], x[i + 1]);
            }
        } else {
#pragma unroll
            for (int i = 0; i < E; ++i) {
                const u32 v = vbase | ((u32)i << NLO);
                const u32 w = ROWS ? cc * R + v : v * C + cc;
                x[i] = sm[swzw<W>(w)];
            }
        }
        if constexpr (FWD)
            fwd_stages<P, KR, K0, 0, XR, OTS, TWM, SCR, SSB, SOT, E>(x, c, t0);
        else
            inv_stages<P, KR, K0, KR - 1, XR, OTS, HAS_S0, TWM, SCR, SSB, SOT, PRE, E>(x, c, t0);
        if constexpr (CANON > 0) {
#pragma unroll
            for (int i = 0; i < E; ++i) x[i] = canon<CANON>(x[i], c.q, c.rc, c.rsh);
        }
        if constexpr (PAIRS) {
#pragma unroll
            for (int i = 0; i < E; i += 2) {
                const u32 w = cc * R + vbase + (u32)i;
                store_pair(sm + swzw<W>(w), x[i], x[i + 1]);
            }
        } else {
#pragma unroll
            for (int i = 0; i < E; ++i) {
                const u32 v = vbase | ((u32)i << NLO);
                const u32 w = ROWS ? cc * R + v : v * C + cc;
                sm[swzw<W>(w)] = x[i];
            }
        }
    }
}

// Range of the values entering round r.
template <int P, int KMAX, bool FWD, int XIN, int r>
__host__ __device__ constexpr int round_in_range()
{
    if constexpr (FWD) return ct_range_after(XIN, rstart(P, KMAX, r));
    else return gs_range_after(XIN, P - rstart(P, KMAX, r) - rsize(P, KMAX, r));
}

// Run all P stages of one tile held in shared memory (rounds separated by
// block barriers; no barrier after the last round).
struct NoHook {
    __device__ __forceinline__ void operator()() const {}
};

// Whether the items of a row tile stay in one warp across the rounds: every
// round has the same radix, each thread holds one item per round, and a
// row's items fit one warp.  The rounds of such a tile exchange data within
// warps only, so a warp barrier separates them instead of a block barrier.
template <int P, int LOGC, int KMAX, int NT>
__host__ __device__ constexpr bool rows_stay_in_warp()
{
    constexpr int nr = nrounds(P, KMAX);
    bool same = true;
    for (int r = 1; r < nr; ++r) same = same && rsize(P, KMAX, r) == rsize(P, KMAX, 0);
    constexpr int per_row = 1 << (P - rsize(P, KMAX, 0));
    return same && per_row <= 32 && (32 % per_row) == 0 && ((1 << LOGC) * per_row) == NT;
}

// Barrier between rounds: the whole block, or (NAMED) named barrier 1 over
// the NT compute threads only (when other warps of the block do not take
// part), or (WARPX) the warp alone.
template <int NT, bool NAMED, bool WARPX = false>
__device__ __forceinline__ void round_barrier()
{
    if constexpr (WARPX)
        __syncwarp();
    else if constexpr (NAMED)
        asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
    else
        __syncthreads();
}

// Twiddle staging of a row tile of the fused kernel (STAGE > 0): the table
// runs of the tile's SCR rows in shared memory.  STAGE 1: round 0's runs in
// `tw` (the tile buffer's own twiddle area), the later rounds' runs and the
// OT factors in `htw`; STAGE 2: all of them in `htw`.  Layout of htw: the
// runs of stages [SSB, P - OTS) (SSB = 0 for STAGE 2, the first stage of
// round 1 for STAGE 1), then the A factors A[2^(P-OTS), 2^P), then the B
// factors, OTS runs of SCR rows.
template <int P, int CR, int KMAX, int OTS, int STAGE>
struct RowStaging {
    static constexpr int KR0 = rsize(P, KMAX, 0);
    static constexpr int SSB = STAGE == 1 ? KR0 : 0;                   // first stage in htw
    static constexpr int N0 = STAGE == 1 ? CR * ((1 << KR0) - 1) : 0;  // entries in the tile buffer
    static constexpr int NT_H = CR * ((1 << (P - OTS)) - (1 << SSB)); // table entries in htw
    static constexpr int NA = OTS ? (1 << P) - (1 << (P - OTS)) : 0;
    static constexpr int NB = OTS * CR;
    static constexpr int A_OFF = NT_H, B_OFF = NT_H + NA;
    static constexpr int NH = NT_H + NA + NB;                          // entries in htw
};

// `mid` runs (in every thread) after the first round executed, before the
// barrier that follows it.  With row staging, `hw` runs before the first
// round that reads htw and `ha` after the last one (wait for the buffer to be
// filled, report it read).
template <int P, int LOGC, int KMAX, bool ROWS, bool FWD, int XIN, bool FINAL, bool HAS_S0, int OTS,
          bool TW_SMEM, int NT, class Hook = NoHook, bool NAMED = false, bool PRELOAD_TW = false, class W = u64,
          int STAGE = 0, bool WARPX = false, class HW = NoHook, class HA = NoHook, bool TBL_LAST = false>
__device__ __forceinline__ void compute_tile(W* sm, const typename WordTypes<W>::Prime& pr,
                                             const typename WordTypes<W>::Tw* tw,
                                             const typename WordTypes<W>::Tw* ota,
                                             const typename WordTypes<W>::Tw* otb, const u32 u_base, const u32 s0,
                                             const u32 tid, Hook mid = Hook(),
                                             const typename WordTypes<W>::Tw* htw = nullptr, HW hw = HW(),
                                             HA ha = HA(), const typename WordTypes<W>::Tw* twg = nullptr)
{
    constexpr int NR = nrounds(P, KMAX);
    static_assert(NR <= 4, "at most four rounds per pass");
    static_assert(FWD ? ct_range_max(XIN, P) <= 16 : gs_range_max(XIN, P) <= 8, "lazy range");
    static_assert(STAGE == 0 || (ROWS && NR >= 2), "row staging needs a row pass of two rounds or more");
    using RS = RowStaging<P, 1 << LOGC, KMAX, OTS, STAGE>;
    constexpr int CRS = 1 << LOGC;
    ItemCtxT<W> c;
    c.q = pr.q;
    c.q4 = pr.q << 2;
    c.rc = pr.rc;
    c.rsh = pr.rsh;
    c.u = u_base;
    c.ubase = u_base;
    c.hi = 0;
    c.s0 = s0;
    c.ninv = pr.ninv;
    c.w1ninv = pr.w1ninv;
    c.tw = tw;
    c.twg = twg;
    c.ota = STAGE ? htw + RS::A_OFF : ota;
    c.otb = STAGE ? htw + RS::B_OFF : otb;
    (void)CRS;

    // per round: where its table twiddles come from
    constexpr int TWM_PLAIN = TW_SMEM ? TW_PASS : TW_GLOBAL;
    constexpr int TWM0 = STAGE ? TW_STAGED : TWM_PLAIN;
    constexpr int TWM1 = STAGE ? TW_STAGED : TWM_PLAIN;
    constexpr int SB0 = 0, SB1 = RS::SSB;
    constexpr int SOT = TBL_LAST ? 2 : (STAGE ? 1 : 0);
    static_assert(!TBL_LAST || (STAGE && OTS == 1), "TBL_LAST takes the staging layout of one OT stage");
    constexpr bool PRE = PRELOAD_TW && !STAGE;
    ItemCtxT<W> c1 = c;
    if constexpr (STAGE) {
        c1.tw = htw;
        if constexpr (STAGE == 2) c.tw = htw;
    }

    // canonical output written by the last round executed
    constexpr int FWD_OUT = ct_range_after(XIN, P);
    constexpr int CANON_FWD = FINAL ? FWD_OUT : 0;
    constexpr int CANON_INV = FINAL ? (HAS_S0 ? 4 : gs_range_after(XIN, P)) : 0;

    if constexpr (FWD) {
        if constexpr (STAGE == 2) hw();
        run_round<P, LOGC, KMAX, 0, ROWS, true, round_in_range<P, KMAX, true, XIN, 0>(), OTS, false,
                  (NR == 1 ? CANON_FWD : 0), TWM0, CRS, SB0, SOT, NT, false>(sm, c, u_base, tid);
        mid();
        if constexpr (NR > 1) {
            round_barrier<NT, NAMED, WARPX>();
            if constexpr (STAGE == 1) hw();
            run_round<P, LOGC, KMAX, 1, ROWS, true, round_in_range<P, KMAX, true, XIN, 1>(), OTS, false,
                      (NR == 2 ? CANON_FWD : 0), TWM1, CRS, SB1, SOT, NT, false>(sm, c1, u_base, tid);
            if constexpr (STAGE && NR == 2) ha();
        }
        if constexpr (NR > 2) {
            round_barrier<NT, NAMED, WARPX>();
            run_round<P, LOGC, KMAX, 2, ROWS, true, round_in_range<P, KMAX, true, XIN, 2>(), OTS, false,
                      (NR == 3 ? CANON_FWD : 0), TWM1, CRS, SB1, SOT, NT, false>(sm, c1, u_base, tid);
            if constexpr (STAGE && NR == 3) ha();
        }
        if constexpr (NR > 3) {
            round_barrier<NT, NAMED, WARPX>();
            run_round<P, LOGC, KMAX, 3, ROWS, true, round_in_range<P, KMAX, true, XIN, 3>(), OTS, false,
                      CANON_FWD, TWM1, CRS, SB1, SOT, NT, false>(sm, c1, u_base, tid);
            if constexpr (STAGE) ha();
        }
    } else {
        if constexpr (STAGE) hw();
        if constexpr (NR > 3) {
            run_round<P, LOGC, KMAX, 3, ROWS, false, round_in_range<P, KMAX, false, XIN, 3>(), OTS, false, 0, TWM1,
                      CRS, SB1, SOT, NT, PRE>(sm, c1, u_base, tid);
            if constexpr (NR == 4) mid();
            round_barrier<NT, NAMED, WARPX>();
        }
        if constexpr (NR > 2) {
            run_round<P, LOGC, KMAX, 2, ROWS, false, round_in_range<P, KMAX, false, XIN, 2>(), OTS, false, 0, TWM1,
                      CRS, SB1, SOT, NT, PRE>(sm, c1, u_base, tid);
            if constexpr (NR == 3) mid();
            round_barrier<NT, NAMED, WARPX>();
        }
        if constexpr (NR > 1) {
            run_round<P, LOGC, KMAX, 1, ROWS, false, round_in_range<P, KMAX, false, XIN, 1>(), OTS, false, 0, TWM1,
                      CRS, SB1, SOT, NT, PRE>(sm, c1, u_base, tid);
            if constexpr (STAGE == 1) ha();
            if constexpr (NR == 2) mid();
            round_barrier<NT, NAMED, WARPX>();
        }
        run_round<P, LOGC, KMAX, 0, ROWS, false, round_in_range<P, KMAX, false, XIN, 0>(), OTS, HAS_S0, CANON_INV,
                  TWM0, CRS, SB0, SOT, NT, PRE>(sm, c, u_base, tid);
        if constexpr (STAGE == 2) ha();
        if constexpr (NR == 1) mid();
    }
}

// ------------------------------------------------------------------ pass ---
// Template parameters:
//   P, LOGC, KMAX, ROWS : geometry (see the file comment)
//   FWD                 : forward (Cooley-Tukey) or inverse (Gentleman-Sande)
//   XIN                 : bound (in units of q) of the values entering the pass
//   FINAL               : the last pass executed: write canonical residues
//   HAS_S0              : the pass holds global stage 0 (s0 == 0)
//   OTS                 : the last OTS stages of the pass use on-the-fly twiddles
//   TW_SMEM             : stage the pass's twiddles Psi[1 .. 2^P) in shared
//                         memory (only when s0 == 0, where they are all it needs)
//   TBL_LAST            : (table plans, OTS 1, staged row twiddles) the last
//                         stage is not factored: its twiddles come from the
//                         table in global memory, the others' runs are staged
// 16-byte global <-> shared moves of a tile: one vector holds 16 / sizeof(W)
// words and lands in shared memory as word pairs (the swizzle keeps pairs).
template <class W>
__device__ __forceinline__ void vec_to_smem(W* sm, u32 w, const uint4 v)
{
    if constexpr (sizeof(W) == 8) {
        store_pair(sm + swz(w), ((u64)v.y << 32) | v.x, ((u64)v.w << 32) | v.z);
    } else {
        store_pair(sm + swzw<W>(w), (W)v.x, (W)v.y);
        store_pair(sm + swzw<W>(w + 2), (W)v.z, (W)v.w);
    }
}
template <class W>
__device__ __forceinline__ uint4 vec_from_smem(const W* sm, u32 w)
{
    W a, b, c, d;
    if constexpr (sizeof(W) == 8) {
        load_pair(sm + swz(w), a, b);
        return make_uint4((u32)a, (u32)(a >> 32), (u32)b, (u32)(b >> 32));
    } else {
        load_pair(sm + swzw<W>(w), a, b);
        load_pair(sm + swzw<W>(w + 2), c, d);
        return make_uint4(a, b, c, d);
    }
}

// 16-byte global -> shared copy that does not pass through registers
// (cp.async, cached in L2 only), and the wait for all of this thread's copies.
__device__ __forceinline__ void cp_async16(void* dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((u32)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Whether a second-pass row tile of the per-pass kernel stages its twiddles
// in shared memory (all table runs of its rows and the OT factors, the
// layout of RowStaging with STAGE 2), so that its rounds read no twiddle
// from global memory: 64-bit words, two rounds or more, and at most 80 KB
// of shared memory with the tile (two or more CTAs per SM).
template <int P, int LOGC, int KMAX, bool ROWS, bool HAS_S0, int OTS, class W>
__host__ __device__ constexpr bool pass_stages_rows()
{
    return ROWS && !HAS_S0 && sizeof(W) == 8 && nrounds(P, KMAX) >= 2 &&
           (size_t)(1 << (P + LOGC)) * 8 + (size_t)RowStaging<P, 1 << LOGC, KMAX, OTS, 2>::NH * 16 <= 80 * 1024;
}

// Resident CTAs per SM the pass kernel's registers are sized for: 768
// threads (24 warps; at most 85 registers per thread).
__host__ __device__ constexpr int pass_min_blocks(int threads) { return threads <= 384 ? 768 / threads : 1; }

// COUNT elements copied by T threads (element i by thread i % T): each thread
// issues up to 8 loads before the stores that consume them, so a thread's
// copies cost one memory latency per 8 elements rather than one each.
template <int T, int COUNT, class V, class LD, class ST>
__device__ __forceinline__ void batched_copy(const u32 tid, LD ld, ST st)
{
    constexpr int PER = (COUNT + T - 1) / T;
    constexpr int B = PER < 8 ? PER : 8;
#pragma unroll
    for (int k0 = 0; k0 < PER; k0 += B) {
        V v[B];
#pragma unroll
        for (int k = 0; k < B; ++k) {
            const u32 i = tid + (u32)(k0 + k) * T;
            if (k0 + k < PER && (COUNT % T == 0 || i < (u32)COUNT)) v[k] = ld(i);
        }
#pragma unroll
        for (int k = 0; k < B; ++k) {
            const u32 i = tid + (u32)(k0 + k) * T;
            if (k0 + k < PER && (COUNT % T == 0 || i < (u32)COUNT)) st(i, v[k]);
        }
    }
}

template <int P, int LOGC, int KMAX, bool ROWS, bool FWD, int XIN, bool FINAL, bool HAS_S0,
          int OTS, bool TW_SMEM, class W = u64, bool TBL_LAST = false>
__global__ void __launch_bounds__(pass_threads(P, LOGC, KMAX), pass_min_blocks(pass_threads(P, LOGC, KMAX)))
ntt_pass_kernel(const PassArgsT<W> a)
{
    using TwT = typename WordTypes<W>::Tw;
    using PrimeT = typename WordTypes<W>::Prime;
    constexpr int R = 1 << P, C = 1 << LOGC;
    constexpr int T = pass_threads(P, LOGC, KMAX);
    constexpr int NR = nrounds(P, KMAX);
    constexpr int TILE = R * C;
    // words per 16-byte vector; tiles below 16 bytes move word by word
    constexpr int VW = TILE * (int)sizeof(W) >= 16 ? 16 / (int)sizeof(W) : 1;
    static_assert(NR <= 4, "at most four rounds per pass");
    static_assert(FWD ? ct_range_max(XIN, P) <= 16 : gs_range_max(XIN, P) <= 8, "lazy range");
    static_assert(!TW_SMEM || HAS_S0, "twiddle staging needs s0 == 0");
    static_assert(ROWS || C % VW == 0, "column tiles hold whole vectors");

    extern __shared__ __align__(16) u64 smem_pass[];
    W* sm = reinterpret_cast<W*>(smem_pass);
    // the tile is a multiple of 16 bytes or is at most 8 bytes; round up for the tables
    TwT* sm_tw = reinterpret_cast<TwT*>(smem_pass + (TILE * sizeof(W) + 15) / 16 * 2);   // 2^P entries
    TwT* sm_ota = sm_tw + (TW_SMEM ? R : 0);                                            // 2^P entries
    // second-pass row tiles: the tile's table runs and OT factors (RowStaging
    // layout, STAGE 2) in place of sm_ota
    constexpr bool SR = pass_stages_rows<P, LOGC, KMAX, ROWS, HAS_S0, OTS, W>();
    using RS = RowStaging<P, C, KMAX, OTS, 2>;
    TwT* const htw = sm_ota;
    static_assert(!TBL_LAST || SR, "the last stage reads the global table only with staged row twiddles");

    const u32 tid = threadIdx.x;
    const u32 tile = blockIdx.x;
    const u32 limb = blockIdx.y + a.limb_offset;
    const u32 pi = a.prime_map ? a.prime_map[limb] : limb % a.L;
    const PrimeT pr = a.primes[pi];
    const u32 nb = a.n - a.s0;                       // bits of u's block size
    W* base = a.data + (size_t)limb * ((size_t)1 << a.n);

    // tile origin
    u32 u_base, l0;
    if constexpr (ROWS) {
        u_base = tile * C;
        l0 = 0;
    } else {
        const u32 per_u = (1u << a.b) >> LOGC;
        u_base = tile / per_u;
        l0 = (tile % per_u) * C;
    }

    if constexpr (sizeof(W) == 8 && VW == 2) {
        // global -> shared: every 16-byte piece by cp.async, all in flight
        // at once, then one wait (a tile's swizzle keeps word pairs together)
        if constexpr (TW_SMEM) {
            const TwT* g = a.tw + (size_t)pi * a.tw_len;
#pragma unroll 1
            for (u32 i = tid; i < (u32)R; i += T) cp_async16(&sm_tw[i], &g[i]);
        }
        if constexpr (SR) {
            // stage sl's run for rows [u_base, u_base + C): C << sl entries at
            // offset C (2^sl - 1), ascending (forward) or the mirrored run
            // the inverse reads; then the A factors of the OT stages and one
            // B factor per row and OT stage
            const TwT* tb = a.tw + (size_t)pi * a.tw_len;
#pragma unroll 1
            for (u32 e = tid; e < (u32)RS::NT_H; e += T) {
                const u32 sl = 31u - (u32)__clz((int)(e / (u32)C + 1u));
                const u32 i = e - (u32)C * ((1u << sl) - 1u);
                const u32 st = FWD ? (1u << (a.s0 + sl)) + (u_base << sl)
                                   : (2u << (a.s0 + sl)) - ((u_base + (u32)C) << sl);
                cp_async16(&htw[e], &tb[st + i]);
            }
            if constexpr (OTS > 0 && !TBL_LAST) {
                const TwT* ga = a.ota + (size_t)pi * R + (1u << (P - OTS));
                for (u32 i = tid; i < (u32)RS::NA; i += T) cp_async16(&htw[RS::A_OFF + i], &ga[i]);
                const TwT* gb = a.otb + (size_t)pi * ((size_t)P << a.s0);
                for (u32 e = tid; e < (u32)RS::NB; e += T) {
                    const u32 k = e / (u32)C, r = e % (u32)C;
                    cp_async16(&htw[RS::B_OFF + e], &gb[((size_t)(P - OTS + k) << a.s0) + u_base + r]);
                }
            }
        } else if constexpr (OTS > 0) {
            const TwT* g = a.ota + (size_t)pi * R;
            for (u32 i = tid; i < (u32)R; i += T) cp_async16(&sm_ota[i], &g[i]);
        }
        if constexpr (ROWS) {
            const W* src = base + ((size_t)u_base << P);
#pragma unroll 1
            for (u32 i = tid; i < (u32)(TILE / 2); i += T) cp_async16(sm + swz(2u * i), src + 2u * i);
        } else {
            constexpr int VPR = C / 2;                    // vectors per row
            const W* blk = base + ((size_t)u_base << nb) + l0;
#pragma unroll 1
            for (u32 i = tid; i < (u32)(TILE / 2); i += T) {
                const u32 v = i / VPR, cv = i % VPR;
                cp_async16(sm + swz(v * C + 2u * cv), blk + ((size_t)v << a.b) + 2u * cv);
            }
        }
        cp_async_wait_all();
    } else {
    // global -> shared, every copy batched (loads in flight before their stores)
    if constexpr (TW_SMEM) {
        const TwT* g = a.tw + (size_t)pi * a.tw_len;
        batched_copy<T, R, TwT>(tid, [&](u32 i) { return g[i]; }, [&](u32 i, const TwT& v) { sm_tw[i] = v; });
    }
    if constexpr (OTS > 0) {
        const TwT* g = a.ota + (size_t)pi * R;
        batched_copy<T, R, TwT>(tid, [&](u32 i) { return g[i]; }, [&](u32 i, const TwT& v) { sm_ota[i] = v; });
    }
    if constexpr (VW == 1) {
        const W* src = base + ((size_t)u_base << P);
        batched_copy<T, TILE, W>(tid, [&](u32 i) { return src[i]; }, [&](u32 i, const W& v) { sm[swzw<W>(i)] = v; });
    } else if constexpr (ROWS) {
        const uint4* src = reinterpret_cast<const uint4*>(base + ((size_t)u_base << P));
        batched_copy<T, TILE / VW, uint4>(tid, [&](u32 i) { return src[i]; },
                                         [&](u32 i, const uint4& v) { vec_to_smem(sm, VW * i, v); });
    } else {
        constexpr int VPR = C / VW;                   // vectors per row
        const W* blk = base + ((size_t)u_base << nb) + l0;
        batched_copy<T, TILE / VW, uint4>(
            tid,
            [&](u32 i) {
                const u32 v = i / VPR, cv = i % VPR;
                return *reinterpret_cast<const uint4*>(blk + ((size_t)v << a.b) + VW * cv);
            },
            [&](u32 i, const uint4& x) { vec_to_smem(sm, (i / VPR) * C + VW * (i % VPR), x); });
    }
    }
    __syncthreads();

    if constexpr (SR)
        compute_tile<P, LOGC, KMAX, ROWS, FWD, XIN, FINAL, HAS_S0, OTS, false, T, NoHook, false, false, W, 2,
                     rows_stay_in_warp<P, LOGC, KMAX, T>(), NoHook, NoHook, TBL_LAST>(
            sm, pr, htw, nullptr, nullptr, u_base, a.s0, tid, NoHook(), htw, NoHook(), NoHook(),
            a.tw + (size_t)pi * a.tw_len);
    else
        compute_tile<P, LOGC, KMAX, ROWS, FWD, XIN, FINAL, HAS_S0, OTS, TW_SMEM, T>(
            sm, pr, TW_SMEM ? sm_tw : a.tw + (size_t)pi * a.tw_len, sm_ota,
            a.otb ? a.otb + (size_t)pi * ((size_t)P << a.s0) : nullptr, u_base, a.s0, tid);
    __syncthreads();

    // shared -> global
    if constexpr (VW == 1) {
        W* dst = base + ((size_t)u_base << P);
        for (u32 i = tid; i < (u32)TILE; i += T) dst[i] = sm[swzw<W>(i)];
    } else if constexpr (ROWS) {
        uint4* dst = reinterpret_cast<uint4*>(base + ((size_t)u_base << P));
        for (u32 i = tid; i < TILE / VW; i += T) dst[i] = vec_from_smem(sm, VW * i);
    } else {
        constexpr int VPR = C / VW;
        W* blk = base + ((size_t)u_base << nb) + l0;
        for (u32 i = tid; i < TILE / VW; i += T) {
            const u32 v = i / VPR, cv = i % VPR;
            *reinterpret_cast<uint4*>(blk + ((size_t)v << a.b) + VW * cv) = vec_from_smem(sm, v * C + VW * cv);
        }
    }
}

template <int P, int LOGC, int KMAX, bool ROWS, bool HAS_S0, bool TW_SMEM, int OTS, class W = u64>
__host__ __device__ constexpr size_t pass_smem_bytes()
{
    constexpr size_t tw = sizeof(typename WordTypes<W>::Tw);
    constexpr size_t base = ((size_t)(1 << (P + LOGC)) * sizeof(W) + 15) / 16 * 16 + (TW_SMEM ? (size_t)(1 << P) * tw : 0);
    if constexpr (pass_stages_rows<P, LOGC, KMAX, ROWS, HAS_S0, OTS, W>())
        return base + (size_t)RowStaging<P, 1 << LOGC, KMAX, OTS, 2>::NH * tw;
    else
        return base + (OTS > 0 ? (size_t)(1 << P) * tw : 0);
}

}  // namespace ntt

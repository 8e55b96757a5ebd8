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
struct ItemCtx {
    const Tw* tw;        // twiddle table base for this prime (smem or global)
    const Tw* ota;       // OT A factors for this prime (smem)
    const Tw* otb;       // OT B factors for this prime (global)
    u64 q, q4;
    u32 mbar;
    u32 u;               // upper index bits (which 2^{n-s0} block)
    u32 hi;              // bits of v above the round digit
    u32 s0;              // first stage of the pass
    Tw ninv, w1ninv;
};

// ---------------------------------------------------------------- forward --
template <int P, int KR, int K0, int k, int X, int OTS, bool TWG, int E>
__device__ __forceinline__ void fwd_stages(u64 (&x)[E], const ItemCtx& c)
{
    if constexpr (k < KR) {
        constexpr int half = E >> (k + 1);
        constexpr int sl = K0 + k;                  // stage within the pass
        constexpr bool ot = sl >= P - OTS;
#pragma unroll
        for (int pre = 0; pre < (1 << k); ++pre) {
            const u32 jlo = ((u32)pre << K0) | c.hi;      // twiddle slot, see tw_slot
            if constexpr (ot) {
                const Tw f1 = c.otb[((u32)sl << c.s0) + c.u];
                const Tw f2 = c.ota[(1u << sl) + jlo];
#pragma unroll
                for (int i = 0; i < half; ++i)
                    ct_bfly_ot<X>(x[pre * 2 * half + i], x[pre * 2 * half + i + half], f1, f2, c.q, c.q4, c.mbar);
            } else {
                const u32 idx = TWG ? (1u << (c.s0 + sl)) + (c.u << sl) + jlo : (1u << sl) + jlo;
                const Tw t = c.tw[idx];
#pragma unroll
                for (int i = 0; i < half; ++i)
                    ct_bfly<X>(x[pre * 2 * half + i], x[pre * 2 * half + i + half], t.w, t.wp, c.q, c.q4, c.mbar);
            }
        }
        fwd_stages<P, KR, K0, k + 1, ct_next(X), OTS, TWG, E>(x, c);
    }
}

// ---------------------------------------------------------------- inverse --
// Stages run from KR-1 down to 0.  HAS_S0: this round holds global stage 0
// (K0 == 0 and s0 == 0), whose butterfly also applies N^{-1}.
template <int P, int KR, int K0, int k, int X, int OTS, bool HAS_S0, bool TWG, int E>
__device__ __forceinline__ void inv_stages(u64 (&x)[E], const ItemCtx& c)
{
    if constexpr (k >= 0) {
        constexpr int half = E >> (k + 1);
        constexpr int sl = K0 + k;
        constexpr bool ot = sl >= P - OTS;
        static_assert(X <= 8, "GS inputs must stay below 8q");
        if constexpr (HAS_S0 && K0 == 0 && k == 0) {
            // global stage 0: a single twiddle Psi^{-1}[1] = -Psi[1]
#pragma unroll
            for (int i = 0; i < half; ++i)
                gs_bfly_scaled<X, true>(x[i], x[i + half], c.w1ninv, c.ninv, c.q);
        } else {
#pragma unroll
            for (int pre = 0; pre < (1 << k); ++pre) {
                const u32 jlo = ((u32)pre << K0) | c.hi;  // twiddle slot, see tw_slot
                if constexpr (ot) {
                    const Tw f1 = c.otb[((u32)sl << c.s0) + c.u];
                    const Tw f2 = c.ota[(1u << sl) + jlo];
#pragma unroll
                    for (int i = 0; i < half; ++i)
                        gs_bfly_ot<X, false>(x[pre * 2 * half + i], x[pre * 2 * half + i + half], f1, f2, c.q, c.mbar);
                } else {
                    // Psi^{-1}[2^s + j] = -Psi[2^{s+1} - 1 - j]
                    const u32 j = TWG ? (c.u << sl) + jlo : jlo;
                    const u32 idx = TWG ? (2u << (c.s0 + sl)) - 1u - j : (2u << sl) - 1u - j;
                    const Tw t = c.tw[idx];
#pragma unroll
                    for (int i = 0; i < half; ++i)
                        gs_bfly<X, true>(x[pre * 2 * half + i], x[pre * 2 * half + i + half], t.w, t.wp, c.q, c.mbar);
                }
            }
        }
        inv_stages<P, KR, K0, k - 1, gs_next(X), OTS, HAS_S0, TWG, E>(x, c);
    }
}

// ------------------------------------------------------------------ round --
// One round: every item of the tile reads its 2^KR elements from shared
// memory, runs KR stages in registers and writes them back.
template <int P, int LOGC, int KMAX, int r, bool ROWS, bool FWD, int XR, int OTS,
          bool HAS_S0, int CANON, bool TWG, int NT>
__device__ __forceinline__ void run_round(u64* sm, ItemCtx c, const u32 u_base, const u32 tid)
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
        u64 x[E];
        if constexpr (PAIRS) {
#pragma unroll
            for (int i = 0; i < E; i += 2) {
                const u32 w = cc * R + vbase + (u32)i;
                const ulonglong2 p = *reinterpret_cast<const ulonglong2*>(sm + swz(w));
                x[i] = p.x;
                x[i + 1] = p.y;
            }
        } else {
#pragma unroll
            for (int i = 0; i < E; ++i) {
                const u32 v = vbase | ((u32)i << NLO);
                const u32 w = ROWS ? cc * R + v : v * C + cc;
                x[i] = sm[swz(w)];
            }
        }
        if constexpr (FWD)
            fwd_stages<P, KR, K0, 0, XR, OTS, TWG, E>(x, c);
        else
            inv_stages<P, KR, K0, KR - 1, XR, OTS, HAS_S0, TWG, E>(x, c);
        if constexpr (CANON > 0) {
#pragma unroll
            for (int i = 0; i < E; ++i) x[i] = canon<CANON>(x[i], c.q, c.mbar);
        }
        if constexpr (PAIRS) {
#pragma unroll
            for (int i = 0; i < E; i += 2) {
                const u32 w = cc * R + vbase + (u32)i;
                *reinterpret_cast<ulonglong2*>(sm + swz(w)) = make_ulonglong2(x[i], x[i + 1]);
            }
        } else {
#pragma unroll
            for (int i = 0; i < E; ++i) {
                const u32 v = vbase | ((u32)i << NLO);
                const u32 w = ROWS ? cc * R + v : v * C + cc;
                sm[swz(w)] = x[i];
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

// Barrier between rounds: the whole block, or (NAMED) named barrier 1 over
// the NT compute threads only (when other warps of the block do not take part).
template <int NT, bool NAMED>
__device__ __forceinline__ void round_barrier()
{
    if constexpr (NAMED)
        asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
    else
        __syncthreads();
}

// `mid` runs (in every thread) after the first round executed, before the
// barrier that follows it.
template <int P, int LOGC, int KMAX, bool ROWS, bool FWD, int XIN, bool FINAL, bool HAS_S0, int OTS,
          bool TW_SMEM, int NT, class Hook = NoHook, bool NAMED = false>
__device__ __forceinline__ void compute_tile(u64* sm, const PrimeDev& pr, const Tw* tw, const Tw* ota,
                                             const Tw* otb, const u32 u_base, const u32 s0, const u32 tid,
                                             Hook mid = Hook())
{
    constexpr int NR = nrounds(P, KMAX);
    static_assert(NR <= 4, "at most four rounds per pass");
    static_assert(FWD ? ct_range_max(XIN, P) <= 16 : gs_range_max(XIN, P) <= 8, "lazy range");
    ItemCtx c;
    c.q = pr.q;
    c.q4 = pr.q << 2;
    c.mbar = pr.mbar;
    c.u = u_base;
    c.hi = 0;
    c.s0 = s0;
    c.ninv = pr.ninv;
    c.w1ninv = pr.w1ninv;
    c.tw = tw;
    c.ota = ota;
    c.otb = otb;

    // canonical output written by the last round executed
    constexpr int FWD_OUT = ct_range_after(XIN, P);
    constexpr int CANON_FWD = FINAL ? FWD_OUT : 0;
    constexpr int CANON_INV = FINAL ? (HAS_S0 ? 4 : gs_range_after(XIN, P)) : 0;

    if constexpr (FWD) {
        run_round<P, LOGC, KMAX, 0, ROWS, true, round_in_range<P, KMAX, true, XIN, 0>(), OTS, false,
                  (NR == 1 ? CANON_FWD : 0), !TW_SMEM, NT>(sm, c, u_base, tid);
        mid();
        if constexpr (NR > 1) {
            round_barrier<NT, NAMED>();
            run_round<P, LOGC, KMAX, 1, ROWS, true, round_in_range<P, KMAX, true, XIN, 1>(), OTS, false,
                      (NR == 2 ? CANON_FWD : 0), !TW_SMEM, NT>(sm, c, u_base, tid);
        }
        if constexpr (NR > 2) {
            round_barrier<NT, NAMED>();
            run_round<P, LOGC, KMAX, 2, ROWS, true, round_in_range<P, KMAX, true, XIN, 2>(), OTS, false,
                      (NR == 3 ? CANON_FWD : 0), !TW_SMEM, NT>(sm, c, u_base, tid);
        }
        if constexpr (NR > 3) {
            round_barrier<NT, NAMED>();
            run_round<P, LOGC, KMAX, 3, ROWS, true, round_in_range<P, KMAX, true, XIN, 3>(), OTS, false,
                      CANON_FWD, !TW_SMEM, NT>(sm, c, u_base, tid);
        }
    } else {
        if constexpr (NR > 3) {
            run_round<P, LOGC, KMAX, 3, ROWS, false, round_in_range<P, KMAX, false, XIN, 3>(), OTS, false, 0, !TW_SMEM, NT>(
                sm, c, u_base, tid);
            if constexpr (NR == 4) mid();
            round_barrier<NT, NAMED>();
        }
        if constexpr (NR > 2) {
            run_round<P, LOGC, KMAX, 2, ROWS, false, round_in_range<P, KMAX, false, XIN, 2>(), OTS, false, 0, !TW_SMEM, NT>(
                sm, c, u_base, tid);
            if constexpr (NR == 3) mid();
            round_barrier<NT, NAMED>();
        }
        if constexpr (NR > 1) {
            run_round<P, LOGC, KMAX, 1, ROWS, false, round_in_range<P, KMAX, false, XIN, 1>(), OTS, false, 0, !TW_SMEM, NT>(
                sm, c, u_base, tid);
            if constexpr (NR == 2) mid();
            round_barrier<NT, NAMED>();
        }
        run_round<P, LOGC, KMAX, 0, ROWS, false, round_in_range<P, KMAX, false, XIN, 0>(), OTS, HAS_S0,
                  CANON_INV, !TW_SMEM, NT>(sm, c, u_base, tid);
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
template <int P, int LOGC, int KMAX, bool ROWS, bool FWD, int XIN, bool FINAL, bool HAS_S0,
          int OTS, bool TW_SMEM>
__global__ void __launch_bounds__(pass_threads(P, LOGC, KMAX))
ntt_pass_kernel(const PassArgs a)
{
    constexpr int R = 1 << P, C = 1 << LOGC;
    constexpr int T = pass_threads(P, LOGC, KMAX);
    constexpr int NR = nrounds(P, KMAX);
    constexpr int TILE = R * C;
    static_assert(NR <= 4, "at most four rounds per pass");
    static_assert(FWD ? ct_range_max(XIN, P) <= 16 : gs_range_max(XIN, P) <= 8, "lazy range");
    static_assert(!TW_SMEM || HAS_S0, "twiddle staging needs s0 == 0");

    extern __shared__ __align__(16) u64 smem[];
    u64* sm = smem;
    Tw* sm_tw = reinterpret_cast<Tw*>(smem + TILE);               // 2^P entries
    Tw* sm_ota = sm_tw + (TW_SMEM ? R : 0);                        // 2^P entries

    const u32 tid = threadIdx.x;
    const u32 tile = blockIdx.x;
    const u32 limb = blockIdx.y + a.limb_offset;
    const u32 pi = a.prime_map ? a.prime_map[limb] : limb % a.L;
    const PrimeDev pr = a.primes[pi];
    const u32 nb = a.n - a.s0;                       // bits of u's block size
    u64* base = a.data + (size_t)limb * ((size_t)1 << a.n);

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

    if constexpr (TW_SMEM) {
        const Tw* g = a.tw + (size_t)pi * a.tw_len;
        for (u32 i = tid; i < (u32)R; i += T) sm_tw[i] = g[i];
    }
    if constexpr (OTS > 0) {
        const Tw* g = a.ota + (size_t)pi * R;
        for (u32 i = tid; i < (u32)R; i += T) sm_ota[i] = g[i];
    }

    // global -> shared (16-byte vectors)
    if constexpr (ROWS) {
        const ulonglong2* src = reinterpret_cast<const ulonglong2*>(base + ((size_t)u_base << P));
        for (u32 i = tid; i < TILE / 2; i += T) {
            const ulonglong2 v = src[i];
            *reinterpret_cast<ulonglong2*>(sm + swz(2 * i)) = v;
        }
    } else {
        constexpr int VPR = C / 2;                    // vectors per row
        const u64* blk = base + ((size_t)u_base << nb) + l0;
        for (u32 i = tid; i < TILE / 2; i += T) {
            const u32 v = i / VPR, cv = i % VPR;
            const ulonglong2 val = *reinterpret_cast<const ulonglong2*>(blk + ((size_t)v << a.b) + 2 * cv);
            *reinterpret_cast<ulonglong2*>(sm + swz(v * C + 2 * cv)) = val;
        }
    }
    __syncthreads();

    compute_tile<P, LOGC, KMAX, ROWS, FWD, XIN, FINAL, HAS_S0, OTS, TW_SMEM, T>(
        sm, pr, TW_SMEM ? sm_tw : a.tw + (size_t)pi * a.tw_len, sm_ota,
        a.otb ? a.otb + (size_t)pi * ((size_t)P << a.s0) : nullptr, u_base, a.s0, tid);
    __syncthreads();

    // shared -> global
    if constexpr (ROWS) {
        ulonglong2* dst = reinterpret_cast<ulonglong2*>(base + ((size_t)u_base << P));
        for (u32 i = tid; i < TILE / 2; i += T)
            dst[i] = *reinterpret_cast<const ulonglong2*>(sm + swz(2 * i));
    } else {
        constexpr int VPR = C / 2;
        u64* blk = base + ((size_t)u_base << nb) + l0;
        for (u32 i = tid; i < TILE / 2; i += T) {
            const u32 v = i / VPR, cv = i % VPR;
            *reinterpret_cast<ulonglong2*>(blk + ((size_t)v << a.b) + 2 * cv) =
                *reinterpret_cast<const ulonglong2*>(sm + swz(v * C + 2 * cv));
        }
    }
}

template <int P, int LOGC, int KMAX, bool TW_SMEM, int OTS>
__host__ __device__ constexpr size_t pass_smem_bytes()
{
    return (size_t)(1 << (P + LOGC)) * 8 + (TW_SMEM ? (size_t)(1 << P) * 16 : 0) +
           (OTS > 0 ? (size_t)(1 << P) * 16 : 0);
}

}  // namespace ntt

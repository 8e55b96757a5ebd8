// Both passes of a two-pass transform in one persistent launch (or the four
// passes of a forward and the inverse of its result).
//
// Work unit = one tile of one pass ("phase") of one limb.  Phase 0 of a limb
// has no dependencies; a tile of phase p > 0 may start only after every tile
// of phase p - 1 of its limb has been written back (per-limb counters), so
// limbs cross the pass boundaries through L2 without a grid-wide barrier and
// without a kernel boundary.  A limb whose phase-p tiles are all written back
// is "published" by phase p: appended to that phase's list in publication
// order, and phase-(p+1) tickets are handed out in that order, so a tile waits
// only while no further limb has been published, never for one particular
// slow limb.  One transform has two phases (the forward: column pass, then
// row pass; the inverse: row pass, then column pass); a forward + inverse
// launch has four (forward column, forward row, inverse row, inverse column).
//
// Each CTA is warp-specialised:
//   * NT compute threads transform tiles held in a ring of shared-memory
//     buffers; they only wait for a buffer to be filled ("full" mbarrier) and
//     report it computed ("empty" mbarrier).
//   * one producer thread (its own warp) runs an event loop: it claims units,
//     at most one ahead of the unit being computed (so the last units spread
//     over the CTAs instead of queueing behind a few); it loads tiles by TMA
//     (2-D tensor maps with the 128-byte swizzle the compute rounds expect),
//     together with the prime's constants and, for column tiles, the
//     twiddles Psi[0, R1) of the column pass; it stores computed tiles by TMA
//     and, once a store has completed, publishes it on its limb's counter.
//
// Claims: (1) a ticket of the latest phase whose limb is already published,
// taken by compare-and-swap so that the ticket taken is the one checked
// (later phases first: limbs finish, and leave L2, before new ones start);
// (2) else a phase-0 ticket, which never waits; (3) else, once every ticket
// of the phases below p is taken, a phase-p ticket, held until its limb is
// published.  Deadlock freedom: a held ticket waits only for tiles of the
// phase below, all of which are then claimed by CTAs that either compute them
// or hold a ticket of a still lower phase, and phase 0 never waits; a CTA that
// holds a ticket keeps storing and publishing its own finished tiles.  Every
// wait is bounded; a wait that runs out sets the plan's status word and the
// CTA stops.  (A CPU simulation of this protocol under random interleavings
// checks these claims.)
//
// Twiddles of row tiles (64-bit words): where they fit, the producer stages
// them in shared memory - round 0's table runs in the tile buffer with the
// tile, the later rounds' runs and the OT factors in a per-CTA buffer filled
// by bulk copies once the previous row tile has released it - so the compute
// threads read no twiddle from global memory.  Otherwise row tiles read the
// global table, which the producer prefetches into L2 with the tile.
//
// Jobs: one launch may transform several independent arrays ("jobs", up to
// MAXJ), each with its own tensor maps and its own plan tables, all of the
// same size and direction.  Limbs are numbered over the launch (job j owns
// limbs [limb0_j, limb0_j + limbs_j)); tickets, counters and the publication
// orders use that numbering, and the producer finds a limb's job by binary
// search over limb0.
//
// Work area (owned by the caller, zero between launches; fused_ctl_words
// words for NP phases): [p] next ticket of phase p, [NP + p] limbs published
// by phase p (p < NP - 1), [2 NP - 1] CTAs finished, then for each phase
// p < NP - 1 the tiles of each limb written back and the published limbs + 1
// in publication order.  The last CTA to finish zeroes it again.
#pragma once
#include "ntt_pass.cuh"
#include "tma.cuh"

#ifndef NTT_FUSED_THREADS_PER_SM
#define NTT_FUSED_THREADS_PER_SM 576    // resident threads per SM the registers are sized for
#endif
#ifndef NTT_FUSED32_THREADS_PER_SM
#define NTT_FUSED32_THREADS_PER_SM 1088 // the same for 32-bit words (two CTAs of 512 + 32 threads)
#endif

namespace ntt {

// bits of the device status word
enum : u32 { STATUS_DEP_TIMEOUT = 1u, STATUS_TMA_TIMEOUT = 2u };

// One job of a launch: a [batch][L][N] array and the tables of its plan
// (W: the data word, 64 or 32 bits).
template <class W = u64>
struct FusedJobT {
    const typename WordTypes<W>::Prime* primes;  // [L]
    const typename WordTypes<W>::Tw* tw;         // [L][tw_len]
    const typename WordTypes<W>::Tw* ota;        // [L][2^p2]      OT A factors, this direction
    const typename WordTypes<W>::Tw* otb;        // [L][p2 << p1]  OT B factors, this direction
    const typename WordTypes<W>::Tw* ota_inv;    // chained launches: the inverse's OT A factors
    const typename WordTypes<W>::Tw* otb_inv;    // chained launches: the inverse's OT B factors
    const W* mulb;           // inverse, 64-bit words: data *= mulb element-wise
                             // before the first pass (null: no product)
    u32 tw_len;
    u32 L;                   // primes per polynomial (local limb l uses prime l % L)
    u32 limb0;               // first limb of the job in the launch's numbering
    u32 reserved;
};
using FusedJob = FusedJobT<u64>;

// Kernel parameters (passed by value as one __grid_constant__ block, so the
// tensor maps live in parameter space).
template <int MAXJ, class W = u64>
struct FusedParams {
    CUtensorMap mapC[MAXJ];  // column view of each job's data
    CUtensorMap mapR[MAXJ];  // row view of each job's data
    FusedJobT<W> job[MAXJ];
    u32* ctl;                // work area (see the file comment)
    u32* status;             // persistent error word
    u32 njobs;
    u32 limbs;               // all jobs
    u32 max_polls;           // bound of every wait loop
    u32 reserved;
};

template <int P1, int P2, int LOGC_R, int KMAX, class W = u64, int OTS = 0>
struct FusedCfg {
    using TwT = typename WordTypes<W>::Tw;
    using PrimeT = typename WordTypes<W>::Prime;
    static constexpr int R1 = 1 << P1, R2 = 1 << P2, CR = 1 << LOGC_R;
    // a column tile is one 128-byte line wide: 16 words of 64 bits or 32 of 32
    static constexpr int LOGC_COL = sizeof(W) == 8 ? 4 : 5;
    static constexpr int COLW = 1 << LOGC_COL;
    static constexpr int TILE_C = COLW * R1;           // column tile: COLW columns x R1 rows
    static constexpr int TILE_R = CR * R2;             // row tile: CR rows of R2 words
    static constexpr int TILE = TILE_C > TILE_R ? TILE_C : TILE_R;
    static constexpr int TC = pass_threads(P1, LOGC_COL, KMAX);
    static constexpr int TR = pass_threads(P2, LOGC_R, KMAX);
    static constexpr int NT = TC > TR ? TC : TR;       // compute threads
    static constexpr int THREADS = NT + 32;            // + the producer warp
    // per buffer: the tile, the column pass's twiddles Psi[0, R1) (or a row
    // tile's first-round twiddle runs), the prime's constants and the unit
    // descriptor, the first three filled by one mbarrier transaction
    static constexpr size_t TW_OFF = (size_t)TILE * sizeof(W);
    static constexpr size_t PR_OFF = TW_OFF + (size_t)R1 * sizeof(TwT);
    static constexpr size_t DESC_OFF = PR_OFF + sizeof(PrimeT);
    static constexpr size_t BUF = (DESC_OFF + 32 + 1023) / 1024 * 1024;
    // Row tiles stage all their twiddles in shared memory (64-bit words, a row
    // pass of two rounds or more) when a per-CTA buffer for the later rounds'
    // runs and the OT factors fits beside two tile buffers at two CTAs per SM:
    // STAGE 1 with round 0's runs in the tile buffer, STAGE 2 with all runs in
    // the per-CTA buffer.  Otherwise three tile buffers, twiddles from global.
    static constexpr size_t SMEM_TWO_PER_SM = 115712;  // dynamic bytes per CTA at two CTAs per SM
    using RS1 = RowStaging<P2, CR, KMAX, OTS, 1>;
    using RS2 = RowStaging<P2, CR, KMAX, OTS, 2>;
    static constexpr size_t htw_bytes(int nh) { return ((size_t)nh * sizeof(TwT) + 1023) / 1024 * 1024; }
    static constexpr bool STAGE_OK = sizeof(W) == 8 && nrounds(P2, KMAX) >= 2;
    static constexpr bool FIT1 = RS1::N0 <= R1 && 2 * BUF + htw_bytes(RS1::NH) + 1024 <= SMEM_TWO_PER_SM;
    static constexpr bool FIT2 = 2 * BUF + htw_bytes(RS2::NH) + 1024 <= SMEM_TWO_PER_SM;
    static constexpr int STAGE = !STAGE_OK ? 0 : FIT1 ? 1 : FIT2 ? 2 : 0;
    using RS = RowStaging<P2, CR, KMAX, OTS, STAGE>;
    static constexpr size_t HTW_BYTES = STAGE ? htw_bytes(RS::NH) : 0;
    static constexpr int NBUF = STAGE ? 2 : 3;         // ring of tile buffers
    static constexpr size_t HTW_OFF = NBUF * BUF;
    static constexpr size_t SMEM = NBUF * BUF + HTW_BYTES + 1024;
    static constexpr int TPS = sizeof(W) == 8 ? NTT_FUSED_THREADS_PER_SM : NTT_FUSED32_THREADS_PER_SM;
    static constexpr int MIN_CTAS = TPS / THREADS > 1 ? TPS / THREADS : 1;
    // row tiles whose rounds exchange data within warps only
    static constexpr bool ROW_WARPX = rows_stay_in_warp<P2, LOGC_R, KMAX, NT>();
};

// unit descriptor written by the producer into the buffer it fills
struct __align__(16) UnitDesc {
    u32 kind;    // the unit's phase, or KIND_STOP
    u32 limb;    // in the launch's numbering
    u32 tile;
    u32 prime;   // local limb % L of its job
    u32 job;
    u32 local;   // limb within its job
    u32 pad[2];
};
enum : u32 { KIND_STOP = 15u };

// Phases of a launch.  One transform (CHAIN false): phase 0 is the pass
// executed first (the column pass of the forward transform, the row pass of
// the inverse), phase 1 the other.  CHAIN: the forward then the inverse
// transform of the same data in one launch: the forward's column pass, its
// row pass, the inverse's row pass, the inverse's column pass.  A tile of
// phase p > 0 may start once every tile of phase p - 1 of its limb has been
// written back.
template <bool FWD, bool CHAIN>
__host__ __device__ constexpr u32 fused_phases() { return CHAIN ? 4u : 2u; }
template <bool FWD, bool CHAIN>
__host__ __device__ constexpr bool phase_is_col(u32 p) { return CHAIN ? (p == 0 || p == 3) : (FWD ? p == 0 : p == 1); }
template <bool FWD, bool CHAIN>
__host__ __device__ constexpr bool phase_is_fwd(u32 p) { return CHAIN ? p < 2 : FWD; }
// 32-bit words of the work area of a launch of `phases` phases over `limbs` limbs
__host__ __device__ constexpr size_t fused_ctl_words(u32 phases, size_t limbs)
{
    return 2 * (size_t)phases + 2 * (size_t)(phases - 1) * limbs;
}

// all compute threads agree on a flag (named barrier 1 with reduction)
template <int NT>
__device__ __forceinline__ bool compute_any(bool flag)
{
    u32 r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((u32)flag), "n"(NT)
        : "memory");
    return r != 0;
}

// MULB: an inverse whose first pass applies an element-wise product
// (FusedJobT::mulb; 64-bit words only).  CHAIN: the forward then the inverse
// transform in one launch (FWD true; see fused_phases).
template <int P1, int P2, int LOGC_R, int KMAX, bool FWD, int OTS, int MAXJ, class W = u64, bool MULB = false,
          bool CHAIN = false>
__global__ void __launch_bounds__(FusedCfg<P1, P2, LOGC_R, KMAX, W>::THREADS,
                                  FusedCfg<P1, P2, LOGC_R, KMAX, W>::MIN_CTAS)
ntt_fused_kernel(const __grid_constant__ FusedParams<MAXJ, W> a)
{
    static_assert(!CHAIN || (FWD && !MULB), "a chained launch runs the forward, then the inverse, without a product");
    using F = FusedCfg<P1, P2, LOGC_R, KMAX, W, OTS>;
    using TwT = typename F::TwT;
    using PrimeT = typename F::PrimeT;
    using RS = typename F::RS;
    constexpr int NT = F::NT;
    constexpr int NBUF = F::NBUF;
    constexpr int STAGE = F::STAGE;
    constexpr u32 NP = fused_phases<FWD, CHAIN>();
    constexpr u32 UC = F::R2 / F::COLW;     // column tiles per limb
    constexpr u32 UR = F::R1 / F::CR;       // row tiles per limb
    constexpr int X_RF = ct_range_after(1, P1);     // entering the forward's row pass
    constexpr int X_CI = gs_range_after(1, P2);     // entering the inverse's column pass
    constexpr u32 NONE = 0xFFFFFFFFu;
    auto is_col = [](u32 kind) { return phase_is_col<FWD, CHAIN>(kind); };
    auto is_fwd = [](u32 kind) { return phase_is_fwd<FWD, CHAIN>(kind); };
    auto units = [](u32 p) -> u32 { return phase_is_col<FWD, CHAIN>(p) ? UC : UR; };

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    auto buf_tile = [&](int b) { return reinterpret_cast<W*>(smem_raw + b * F::BUF); };
    auto buf_tw = [&](int b) { return reinterpret_cast<TwT*>(smem_raw + b * F::BUF + F::TW_OFF); };
    auto buf_pr = [&](int b) { return reinterpret_cast<PrimeT*>(smem_raw + b * F::BUF + F::PR_OFF); };
    auto buf_desc = [&](int b) { return reinterpret_cast<volatile UnitDesc*>(smem_raw + b * F::BUF + F::DESC_OFF); };
    TwT* const htw = reinterpret_cast<TwT*>(smem_raw + F::HTW_OFF);      // staged row twiddles (STAGE)
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + F::HTW_OFF + F::HTW_BYTES);
    uint64_t* empty = full + NBUF;
    uint64_t* htw_full = empty + NBUF;      // the staged row twiddles have landed
    uint64_t* htw_empty = htw_full + 1;     // the compute threads have read them

    const u32 tid = threadIdx.x;
    if (tid == 0) {
        for (int i = 0; i < NBUF; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], NT);
        }
        mbar_init(htw_full, 1);
        mbar_init(htw_empty, NT);
        fence_mbar_init();
    }
    __syncthreads();

    if (tid >= (u32)NT) {
        if (tid != (u32)NT) return;
        // =================================================== producer ====
        // work area: [p] next ticket of phase p; [NP + p] limbs published by
        // phase p (p < NP - 1); [2 NP - 1] CTAs finished; then per phase
        // p < NP - 1 the tiles of each limb written back and the published
        // limbs + 1 in publication order
        u32* const ctl = a.ctl;
        auto done_of = [&](u32 p) { return ctl + 2 * NP + 2 * p * a.limbs; };
        auto list_of = [&](u32 p) { return ctl + 2 * NP + (2 * p + 1) * a.limbs; };
        u32 issued = 0, stored = 0;             // units loaded / stored by this CTA
        u32 q0 = 0, q1 = 0, q2 = 0, qn = 0;      // committed stores not yet published (FIFO)
        u32 left = (1u << NP) - 1u;              // phases that may still have tickets
        bool stopped = false, failed = false;
        u32 held = NONE, held_p = 0;             // claimed ticket waiting for its limb
        u32 idle = 0;

        // job of a limb of the launch (binary search over limb0)
        auto job_of = [&](u32 limb) -> u32 {
            u32 lo = 0;
            if constexpr (MAXJ > 1) {
                u32 hi = a.njobs;
                while (hi - lo > 1) {
                    const u32 mid = (lo + hi) >> 1;
                    if (a.job[mid].limb0 <= limb) lo = mid;
                    else hi = mid;
                }
            }
            return lo;
        };
        // the i-th limb published by phase p, NONE while unpublished
        auto pub_limb = [&](u32 p, u32 i) -> u32 {
            const u32 v = ld_acquire(&list_of(p)[i]);
            return v ? v - 1u : NONE;
        };
        // a completed store of a tile of phase p < NP - 1 counts for its limb
        auto publish_entry = [&](u32 e) {
            if (e) {
                const u32 p = (e >> 28) - 1u, limb = e & 0x0FFFFFFFu;
                fence_proxy_async_global();
                if (atom_acq_rel_add(&done_of(p)[limb], 1u) == units(p) - 1u) {
                    // this tile completed the limb: append it to the publication order
                    const u32 pos = atomicAdd(&ctl[NP + p], 1u);
                    st_release(&list_of(p)[pos], limb + 1u);
                }
            }
        };
        // publish all committed stores but the newest (their stores are complete)
        auto publish_older = [&]() {
            if (qn >= 2) {
                bulk_wait<1>();
                publish_entry(q0);
                if (qn == 3) publish_entry(q1);
                q0 = qn == 3 ? q2 : q1;
                qn = 1;
            }
        };
        auto publish_all = [&]() {
            if (qn) {
                bulk_wait<0>();
                publish_entry(q0);
                if (qn > 1) publish_entry(q1);
                if (qn > 2) publish_entry(q2);
                qn = 0;
            }
        };
        // first table entry of stage sl's run for rows [u0, u0 + CR), read by
        // the forward (or, mirrored, by the inverse)
        auto run_start = [&](int sl, u32 u0, bool fwd) -> u32 {
            return fwd ? (1u << (P1 + sl)) + (u0 << sl) : (2u << (P1 + sl)) - ((u0 + (u32)F::CR) << sl);
        };
        // row tiles loaded whose staged twiddles are still to be copied into
        // htw (unit numbers, in load order), and the copies issued so far
        u32 hq[NBUF > 1 ? NBUF : 1] = {};
        u32 hq_head = 0, hq_tail = 0, fills = 0;
        (void)hq;
        auto fill_htw = [&]() -> bool {
            if constexpr (STAGE) {
                if (hq_head == hq_tail) return false;
                if (fills && !mbar_test(htw_empty, (fills - 1) & 1u)) return false;
                const volatile UnitDesc* d = buf_desc((int)(hq[hq_head % NBUF] % NBUF));
                const u32 j = MAXJ > 1 ? d->job : 0u, pi = d->prime, u0 = d->tile * (u32)F::CR;
                const bool fwd = is_fwd(d->kind);
                const FusedJobT<W>& J = a.job[j];
                const TwT* base = J.tw + (size_t)pi * J.tw_len;
                mbar_arrive_expect_tx(htw_full, (u32)RS::NH * (u32)sizeof(TwT));
#pragma unroll
                for (int sl = RS::SSB; sl < P2 - OTS; ++sl)
                    bulk_load(htw + F::CR * ((1 << sl) - (1 << RS::SSB)), base + run_start(sl, u0, fwd),
                              ((u32)F::CR << sl) * (u32)sizeof(TwT), htw_full);
                if constexpr (OTS > 0) {
                    const TwT* ota = CHAIN && !fwd ? J.ota_inv : J.ota;
                    const TwT* otb = CHAIN && !fwd ? J.otb_inv : J.otb;
                    bulk_load(htw + RS::A_OFF, ota + (size_t)pi * F::R2 + (1u << (P2 - OTS)),
                              (u32)RS::NA * (u32)sizeof(TwT), htw_full);
#pragma unroll
                    for (int i = 0; i < OTS; ++i)
                        bulk_load(htw + RS::B_OFF + i * F::CR,
                                  otb + (size_t)pi * ((size_t)P2 << P1) + ((size_t)(P2 - OTS + i) << P1) + u0,
                                  (u32)F::CR * (u32)sizeof(TwT), htw_full);
                }
                ++hq_head;
                ++fills;
                return true;
            } else {
                return false;
            }
        };
        auto load = [&](u32 kind, u32 limb, u32 tile) {
            const int b = (int)(issued % NBUF);
            const u32 j = job_of(limb);
            const FusedJobT<W>& J = a.job[j];
            const u32 local = limb - J.limb0, pi = local % J.L;
            volatile UnitDesc* d = buf_desc(b);
            d->kind = kind;
            d->limb = limb;
            d->tile = tile;
            d->prime = pi;
            d->job = j;
            d->local = local;
            // the buffer's previous store has read it.  A unit is claimed with
            // at most one unit unstored, right after a store: with three
            // buffers the buffer's previous store is older than the newest
            // one (wait for all but the newest); with two it is the newest
            bulk_wait_read<NBUF == 2 ? 0 : 1>();
            // a tile of a later phase reads what other CTAs' stores wrote
            if (kind > 0) fence_proxy_async_global();
            W* dst = buf_tile(b);
            if (is_col(kind)) {
                mbar_arrive_expect_tx(&full[b], F::TILE_C * (u32)sizeof(W) + F::R1 * (u32)sizeof(TwT) +
                                                    (u32)sizeof(PrimeT));
                tma_load_2d(dst, &a.mapC[j], (int)(tile * F::COLW), (int)(local * F::R1), &full[b]);
                bulk_load(buf_tw(b), J.tw + (size_t)pi * J.tw_len, F::R1 * (u32)sizeof(TwT), &full[b]);
            } else {
                const bool fwd = is_fwd(kind);
                mbar_arrive_expect_tx(&full[b], F::TILE_R * (u32)sizeof(W) + (u32)sizeof(PrimeT) +
                                                    (u32)RS::N0 * (u32)sizeof(TwT));
                tma_load_2d(dst, &a.mapR[j], 0,
                            (int)(local * (F::R1 * F::R2 / F::COLW) + tile * (F::TILE_R / F::COLW)), &full[b]);
                // table runs of the row pass: stage sl of rows [u0, u0 + CR)
                // reads CR << sl consecutive entries (mirrored for the inverse)
                const TwT* base = J.tw + (size_t)pi * J.tw_len;
                const u32 u0 = tile * (u32)F::CR;
                if constexpr (STAGE == 1) {
                    // round 0's runs into the tile buffer, with the tile
#pragma unroll
                    for (int sl = 0; sl < RS::KR0; ++sl)
                        bulk_load(buf_tw(b) + F::CR * ((1 << sl) - 1), base + run_start(sl, u0, fwd),
                                  ((u32)F::CR << sl) * (u32)sizeof(TwT), &full[b]);
                }
                if constexpr (STAGE) {
                    hq[hq_tail++ % NBUF] = issued;      // the later rounds' runs: when the buffer is free
                } else {
                    // into L2, for the compute threads' loads
#pragma unroll
                    for (int sl = 0; sl < P2 - OTS; ++sl)
                        bulk_prefetch_l2(base + run_start(sl, u0, fwd), ((u32)F::CR << sl) * (u32)sizeof(TwT));
                }
                // the other factor of a fused element-wise product (the inverse's
                // first pass multiplies the tile by it), into L2
                if constexpr (MULB && !FWD && sizeof(W) == 8) {
                    if (J.mulb)
                        bulk_prefetch_l2(J.mulb + (size_t)local * (F::R1 * F::R2) + (size_t)tile * F::TILE_R,
                                         (u32)F::TILE_R * (u32)sizeof(W));
                }
            }
            bulk_load(buf_pr(b), J.primes + pi, (u32)sizeof(PrimeT), &full[b]);
            ++issued;
        };
        // Claim the next unit.  (1) A ticket of the latest phase whose limb is
        // published, taken by compare-and-swap so that the ticket taken is the
        // one checked (later phases first: limbs finish, and their data leaves
        // L2, before new limbs start).  (2) A ticket of phase 0, which never
        // waits.  (3) Once every ticket of the phases below p has been taken,
        // a ticket of phase p, held until its limb is published: the tiles it
        // waits for are then all claimed by CTAs that do not wait for it, so
        // holding cannot deadlock.
        auto claim = [&]() -> bool {
            for (u32 p = NP - 1; p >= 1; --p) {
                if (!((left >> p) & 1u)) continue;
                const u32 tot = a.limbs * units(p);
                const u32 t = ld_relaxed(&ctl[p]);
                if (t >= tot) {
                    left &= ~(1u << p);
                    continue;
                }
                const u32 limb = pub_limb(p - 1, t / units(p));
                if (limb != NONE && atomicCAS(&ctl[p], t, t + 1u) == t) {
                    load(p, limb, t % units(p));
                    return true;
                }
            }
            if (left & 1u) {
                const u32 t = atomicAdd(&ctl[0], 1u);
                if (t < a.limbs * units(0)) {
                    load(0, t / units(0), t % units(0));
                    return true;
                }
                left &= ~1u;
            }
            for (u32 p = 1; p < NP; ++p) {
                if (left & ((1u << p) - 1u)) break;        // a lower phase may still have tickets
                if (!((left >> p) & 1u)) continue;
                const u32 t = atomicAdd(&ctl[p], 1u);
                if (t >= a.limbs * units(p)) {
                    left &= ~(1u << p);
                    continue;
                }
                const u32 limb = pub_limb(p - 1, t / units(p));
                if (limb != NONE) {
                    load(p, limb, t % units(p));
                } else {
                    held = t;
                    held_p = p;
                }
                return true;
            }
            return false;
        };

        for (u32 j = 0; j < a.njobs && j < (u32)MAXJ; ++j) {
            prefetch_tensormap(&a.mapC[j]);
            prefetch_tensormap(&a.mapR[j]);
        }
        for (;;) {
            bool progress = fill_htw();
            // store computed tiles, in order
            while (stored < issued && mbar_test(&empty[stored % NBUF], (stored / NBUF) & 1u)) {
                const int b = (int)(stored % NBUF);
                const volatile UnitDesc* d = buf_desc(b);
                const u32 kind = d->kind, limb = d->limb, tile = d->tile, local = d->local;
                const u32 j = MAXJ > 1 ? d->job : 0u;
                const W* src = buf_tile(b);
                if (is_col(kind))
                    tma_store_2d(&a.mapC[j], (int)(tile * F::COLW), (int)(local * F::R1), src);
                else
                    tma_store_2d(&a.mapR[j], 0, (int)(local * (F::R1 * F::R2 / F::COLW) + tile * (F::TILE_R / F::COLW)),
                                 src);
                bulk_commit();
                const u32 e = kind + 1u < NP ? ((kind + 1u) << 28) | limb : 0u;
                if (qn == 0) q0 = e;
                else if (qn == 1) q1 = e;
                else q2 = e;
                ++qn;
                ++stored;
                publish_older();
                progress = true;
            }
            if (stopped) {
                if (stored + 1 == issued) break;     // every real unit stored (the last slot is the stop)
            } else if (issued - stored < 2u) {
                // nothing but the unit in compute is pending: pick the next unit
                if (held != NONE) {
                    const u32 limb = pub_limb(held_p - 1, held / units(held_p));
                    if (limb != NONE) {
                        load(held_p, limb, held % units(held_p));
                        held = NONE;
                        progress = true;
                    }
                } else {
                    if (claim()) progress = true;
                    if (left == 0 && held == NONE) {
                        // no work left: a stop descriptor in the next buffer
                        const int b = (int)(issued % NBUF);
                        buf_desc(b)->kind = KIND_STOP;
                        mbar_arrive(&full[b]);
                        ++issued;
                        stopped = true;
                        progress = true;
                    }
                }
            }
            if (progress) {
                idle = 0;
                continue;
            }
            // nothing moved: publish what is complete (another limb may wait on it), then wait
            publish_all();
            if (++idle > a.max_polls) {
                failed = true;
                break;
            }
            if (stored < issued && (held == NONE || issued - stored >= 2u) && hq_head == hq_tail) {
                // the only event that can come is the oldest unit's compute
                // finishing: suspend on its barrier (a bounded try_wait)
                // instead of polling, which would take issue slots from the
                // compute warps of this SM sub-partition
                mbar_try_wait(&empty[stored % NBUF], (stored / NBUF) & 1u);
            } else {
                __nanosleep(held != NONE ? 256 : 64);
            }
        }
        publish_all();
        // every copy this producer issued into shared memory has landed (a
        // bounded wait) before the CTA may exit: the last NBUF tile loads and
        // the last staged-twiddle copy
        for (u32 k = issued > (u32)NBUF ? issued - (u32)NBUF : 0u; k < issued; ++k)
            mbar_wait(&full[k % NBUF], (k / NBUF) & 1u, a.max_polls);
        if (STAGE && fills) mbar_wait(htw_full, (fills - 1) & 1u, a.max_polls);
        if (failed) {
            atomicOr(a.status, held != NONE ? STATUS_DEP_TIMEOUT : STATUS_TMA_TIMEOUT);
            if (!stopped && issued - stored < (u32)NBUF) {
                const int b = (int)(issued % NBUF);
                buf_desc(b)->kind = KIND_STOP;
                mbar_arrive(&full[b]);
            }
        }
        // the last CTA to finish zeroes the work area for the next launch
        __threadfence();
        if (atomicAdd(&ctl[2 * NP - 1], 1u) == gridDim.x - 1) {
            const size_t words = fused_ctl_words(NP, a.limbs);
            for (size_t i = 0; i < words; ++i) ctl[i] = 0u;
            __threadfence();
        }
        return;
    }

    // ===================================================== compute ======
    u32 rt = 0;                  // row tiles computed (phase of the staged-twiddle barriers)
    bool htw_lost = false;       // a wait for staged twiddles ran out
    for (u32 k = 0;; ++k) {
        const int b = (int)(k % NBUF);
        const bool got = mbar_wait(&full[b], (k / NBUF) & 1u, a.max_polls);
        if (compute_any<NT>(!got || htw_lost)) {
            if (tid == 0) atomicOr(a.status, STATUS_TMA_TIMEOUT);
            break;
        }
        const u32 kind = buf_desc(b)->kind;
        if (kind == KIND_STOP) break;
        const u32 tile = buf_desc(b)->tile;
        const u32 pi = buf_desc(b)->prime;
        W* sm = buf_tile(b);
        const PrimeT& pr = *buf_pr(b);
        if (is_col(kind)) {
            // column pass: twiddles Psi[0, R1) staged with the tile; the
            // forward's first pass, or the inverse's last (canonical output)
            if (is_fwd(kind))
                compute_tile<P1, F::LOGC_COL, KMAX, false, true, 1, false, true, 0, true, NT, NoHook, true>(
                    sm, pr, buf_tw(b), nullptr, nullptr, 0u, 0u, tid);
            else
                compute_tile<P1, F::LOGC_COL, KMAX, false, false, X_CI, true, true, 0, true, NT, NoHook, true>(
                    sm, pr, buf_tw(b), nullptr, nullptr, 0u, 0u, tid);
        } else {
            // row pass: the forward's last (canonical output), or the inverse's first
            const bool fwd = is_fwd(kind);
            const FusedJobT<W>& J = a.job[MAXJ > 1 ? buf_desc(b)->job : 0u];
            if constexpr (MULB && !FWD && sizeof(W) == 8) {
                // fused element-wise product (Sec. III-A): the tile of the first
                // factor's transform times the second's, canonical, before the
                // inverse stages; the row tile is TILE_R consecutive words of the limb
                if (J.mulb) {
                    const W* bt = J.mulb + (size_t)buf_desc(b)->local * (F::R1 * F::R2) + (size_t)tile * F::TILE_R;
                    for (u32 w = 2u * tid; w < (u32)F::TILE_R; w += 2u * NT) {
                        const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(bt + w);
                        W x0, x1;
                        load_pair(sm + swzw<W>(w), x0, x1);
                        x0 = canon<3>(mulmod_barrett(x0, v.x, pr.q, pr.mu, pr.k), pr.q, pr.rc, pr.rsh);
                        x1 = canon<3>(mulmod_barrett(x1, v.y, pr.q, pr.mu, pr.k), pr.q, pr.rc, pr.rsh);
                        store_pair(sm + swzw<W>(w), x0, x1);
                    }
                    round_barrier<NT, true>();
                }
            }
            if constexpr (STAGE) {
                // all twiddles from shared memory: round 0's runs in the tile
                // buffer (STAGE 1), the rest in htw once the producer's copy
                // has landed; htw is released after the last round reading it
                const u32 ph = rt & 1u;
                auto hw = [&]() {
                    if (!mbar_wait(htw_full, ph, a.max_polls)) htw_lost = true;
                };
                auto ha = [&]() { mbar_arrive(htw_empty); };
                const TwT* tw0 = STAGE == 1 ? buf_tw(b) : htw;
                if (fwd)
                    compute_tile<P2, LOGC_R, KMAX, true, true, X_RF, true, false, OTS, false, NT, NoHook, true, false, W,
                                 STAGE, F::ROW_WARPX>(sm, pr, tw0, nullptr, nullptr, tile * F::CR, (u32)P1, tid,
                                                      NoHook(), htw, hw, ha);
                else
                    compute_tile<P2, LOGC_R, KMAX, true, false, 1, false, false, OTS, false, NT, NoHook, true, false, W,
                                 STAGE, F::ROW_WARPX>(sm, pr, tw0, nullptr, nullptr, tile * F::CR, (u32)P1, tid,
                                                      NoHook(), htw, hw, ha);
                ++rt;
            } else {
                const TwT* tw = J.tw + (size_t)pi * J.tw_len;
                const TwT* ota_t = CHAIN && !fwd ? J.ota_inv : J.ota;
                const TwT* otb_t = CHAIN && !fwd ? J.otb_inv : J.otb;
                const TwT* ota = ota_t ? ota_t + (size_t)pi * F::R2 : nullptr;
                const TwT* otb = otb_t ? otb_t + (size_t)pi * ((size_t)P2 << P1) : nullptr;
                if (fwd)
                    compute_tile<P2, LOGC_R, KMAX, true, true, X_RF, true, false, OTS, false, NT, NoHook, true>(
                        sm, pr, tw, ota, otb, tile * F::CR, (u32)P1, tid);
                else
                    compute_tile<P2, LOGC_R, KMAX, true, false, 1, false, false, OTS, false, NT, NoHook, true,
                                 sizeof(W) == 8>(sm, pr, tw, ota, otb, tile * F::CR, (u32)P1, tid);
            }
        }
        // make this thread's shared-memory writes visible to the TMA store
        fence_proxy_async_shared();
        mbar_arrive(&empty[b]);
    }
}

}  // namespace ntt

// Both passes of a two-pass transform in one persistent launch.
//
// Work unit = one tile of one pass of one limb.  The first-executed pass (A)
// of a limb has no dependencies; a tile of the second pass (B) may start only
// after every A tile of its limb has been written back (per-limb counters), so
// limbs cross the pass boundary through L2 without a grid-wide barrier and
// without a kernel boundary.  A limb whose A tiles are all written back is
// "published": appended to a list in publication order, and B tickets are
// handed out in that order, so a B tile waits only while no further limb has
// been published, never for one particular slow limb.
//
// Each CTA is warp-specialised:
//   * NT compute threads transform tiles held in a ring of three shared-memory
//     buffers; they only wait for a buffer to be filled ("full" mbarrier) and
//     report it computed ("empty" mbarrier).
//   * one producer thread (its own warp) runs an event loop: it claims units
//     from two global queues, at most one unit ahead of the one being
//     computed (so the last units spread over the CTAs instead of queueing
//     behind a few), preferring a B tile whose limb is already published and
//     otherwise taking an A tile, so a CTA never idles on a dependency while
//     other work is left; it loads tiles by TMA (2-D tensor
//     maps with the 128-byte swizzle the compute rounds expect), together
//     with the prime's constants and, for column tiles, the twiddles Psi[0,R1)
//     of the column pass; it stores computed tiles by TMA and, once a store
//     of an A tile has completed, publishes it on the limb's counter.
//
// Order: A tiles are taken first while the A queue is less than a_window
// limbs ahead of the B queue (the host sizes the window so that the
// intermediate results of that many limbs stay in L2); beyond it a B tile
// whose limb is published goes first.  Taking A tiles early keeps the
// dependency waits off the end of the launch.
//
// Row tiles read the twiddles of their second pass from the global table; the
// producer prefetches the runs a row tile will read into L2 when it loads the
// tile, so the compute warps' loads of them hit L2.
//
// Deadlock freedom: A tiles never wait.  A producer holds at most one B tile
// whose limb is not yet published, and while it polls for that limb it keeps
// storing and publishing its own finished tiles, so every A tile that any B
// tile waits for is eventually published.  Every wait is bounded; a wait that
// runs out sets the plan's status word and the CTA stops.
//
// Jobs: one launch may transform several independent arrays ("jobs", up to
// MAXJ), each with its own tensor maps and its own plan tables, all of the
// same size and direction.  Limbs are numbered over the launch (job j owns
// limbs [limb0_j, limb0_j + limbs_j)); tickets, counters and the publication
// order use that numbering, and the producer finds a limb's job by binary
// search over limb0.
//
// Work area (owned by the caller, zero between launches; 4 + 2 * limbs
// words): [0] next A ticket, [1] next B ticket, [2] CTAs finished, [3] limbs
// published, [4 + limb] A tiles of the limb written back, [4 + limbs + i] the
// i-th published limb plus one (0 while not yet published).  The last CTA to
// finish zeroes it again.
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
    u32 a_window;            // limbs the A queue may run ahead before ready B tiles are preferred
    u32 max_polls;           // bound of every wait loop
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
    u32 kind;    // KIND_A, KIND_B or KIND_STOP
    u32 limb;    // in the launch's numbering
    u32 tile;
    u32 prime;   // local limb % L of its job
    u32 job;
    u32 local;   // limb within its job
    u32 pad[2];
};
enum : u32 { KIND_A = 0u, KIND_B = 1u, KIND_STOP = 2u };

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
// (FusedJobT::mulb; 64-bit words only)
template <int P1, int P2, int LOGC_R, int KMAX, bool FWD, int OTS, int MAXJ, class W = u64, bool MULB = false>
__global__ void __launch_bounds__(FusedCfg<P1, P2, LOGC_R, KMAX, W>::THREADS,
                                  FusedCfg<P1, P2, LOGC_R, KMAX, W>::MIN_CTAS)
ntt_fused_kernel(const __grid_constant__ FusedParams<MAXJ, W> a)
{
    using F = FusedCfg<P1, P2, LOGC_R, KMAX, W, OTS>;
    using TwT = typename F::TwT;
    using PrimeT = typename F::PrimeT;
    using RS = typename F::RS;
    constexpr int NT = F::NT;
    constexpr int NBUF = F::NBUF;
    constexpr int STAGE = F::STAGE;
    constexpr u32 UC = F::R2 / F::COLW;     // column tiles per limb
    constexpr u32 UR = F::R1 / F::CR;       // row tiles per limb
    constexpr u32 UA = FWD ? UC : UR, UB = FWD ? UR : UC;
    constexpr int X_B = FWD ? ct_range_after(1, P1) : gs_range_after(1, P2);
    constexpr u32 NONE = 0xFFFFFFFFu;

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

    // an A (first-executed pass) tile is a column tile for the forward
    // transform and a row tile for the inverse
    auto is_col = [](u32 kind) { return FWD ? kind == KIND_A : kind == KIND_B; };

    if (tid >= (u32)NT) {
        if (tid != (u32)NT) return;
        // =================================================== producer ====
        u32* const done = a.ctl + 4;
        u32* const order = a.ctl + 4 + a.limbs;  // published limbs + 1, in publication order
        const u32 totalA = a.limbs * UA, totalB = a.limbs * UB;
        u32 issued = 0, stored = 0;             // units loaded / stored by this CTA
        u32 q0 = 0, q1 = 0, q2 = 0, qn = 0;      // committed stores not yet published (FIFO)
        bool a_left = true, b_left = true, stopped = false, failed = false;
        u32 held = NONE;                         // claimed B ticket waiting for its limb
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

        auto publish_entry = [&](u32 e) {
            if (e & 0x80000000u) {
                const u32 limb = e & 0x7FFFFFFFu;
                fence_proxy_async_global();
                if (atom_acq_rel_add(&done[limb], 1u) == UA - 1u) {
                    // this tile completed the limb: append it to the publication order
                    const u32 pos = atomicAdd(&a.ctl[3], 1u);
                    st_release(&order[pos], limb + 1u);
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
        // first table entry of stage sl's run for rows [u0, u0 + CR)
        auto run_start = [&](int sl, u32 u0) -> u32 {
            return FWD ? (1u << (P1 + sl)) + (u0 << sl) : (2u << (P1 + sl)) - ((u0 + (u32)F::CR) << sl);
        };
        // row tiles loaded whose staged twiddles are still to be copied into
        // htw (unit numbers, in load order), and the copies issued so far
        u32 hq[NBUF > 1 ? NBUF : 1];
        u32 hq_head = 0, hq_tail = 0, fills = 0;
        (void)hq;
        auto fill_htw = [&]() -> bool {
            if constexpr (STAGE) {
                if (hq_head == hq_tail) return false;
                if (fills && !mbar_test(htw_empty, (fills - 1) & 1u)) return false;
                const volatile UnitDesc* d = buf_desc((int)(hq[hq_head % NBUF] % NBUF));
                const u32 j = MAXJ > 1 ? d->job : 0u, pi = d->prime, u0 = d->tile * (u32)F::CR;
                const FusedJobT<W>& J = a.job[j];
                const TwT* base = J.tw + (size_t)pi * J.tw_len;
                mbar_arrive_expect_tx(htw_full, (u32)RS::NH * (u32)sizeof(TwT));
#pragma unroll
                for (int sl = RS::SSB; sl < P2 - OTS; ++sl)
                    bulk_load(htw + F::CR * ((1 << sl) - (1 << RS::SSB)), base + run_start(sl, u0),
                              ((u32)F::CR << sl) * (u32)sizeof(TwT), htw_full);
                if constexpr (OTS > 0) {
                    bulk_load(htw + RS::A_OFF, J.ota + (size_t)pi * F::R2 + (1u << (P2 - OTS)),
                              (u32)RS::NA * (u32)sizeof(TwT), htw_full);
#pragma unroll
                    for (int i = 0; i < OTS; ++i)
                        bulk_load(htw + RS::B_OFF + i * F::CR,
                                  J.otb + (size_t)pi * ((size_t)P2 << P1) + ((size_t)(P2 - OTS + i) << P1) + u0,
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
            // the buffer's previous store has read it: at most one unit is
            // unstored when a unit is claimed, so at most two stores were
            // committed after that one; waiting for all but the newest suffices
            bulk_wait_read<1>();
            if (kind == KIND_B) fence_proxy_async_global();
            W* dst = buf_tile(b);
            if (is_col(kind)) {
                mbar_arrive_expect_tx(&full[b], F::TILE_C * (u32)sizeof(W) + F::R1 * (u32)sizeof(TwT) +
                                                    (u32)sizeof(PrimeT));
                tma_load_2d(dst, &a.mapC[j], (int)(tile * F::COLW), (int)(local * F::R1), &full[b]);
                bulk_load(buf_tw(b), J.tw + (size_t)pi * J.tw_len, F::R1 * (u32)sizeof(TwT), &full[b]);
            } else {
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
                        bulk_load(buf_tw(b) + F::CR * ((1 << sl) - 1), base + run_start(sl, u0),
                                  ((u32)F::CR << sl) * (u32)sizeof(TwT), &full[b]);
                }
                if constexpr (STAGE) {
                    hq[hq_tail++ % NBUF] = issued;      // the later rounds' runs: when the buffer is free
                } else {
                    // into L2, for the compute threads' loads
#pragma unroll
                    for (int sl = 0; sl < P2 - OTS; ++sl)
                        bulk_prefetch_l2(base + run_start(sl, u0), ((u32)F::CR << sl) * (u32)sizeof(TwT));
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
        // limb of B ticket t: the (t / UB)-th published limb, NONE while unpublished
        auto b_limb = [&](u32 t) -> u32 {
            const u32 v = ld_acquire(&order[t / UB]);
            return v ? v - 1u : NONE;
        };
        auto claim_b = [&](bool& claimed) {
            const u32 t = atomicAdd(&a.ctl[1], 1u);
            if (t < totalB) {
                const u32 limb = b_limb(t);
                if (limb != NONE) load(KIND_B, limb, t % UB);
                else held = t;
                claimed = true;
            } else {
                b_left = false;
            }
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
                const u32 e = kind == KIND_A ? (0x80000000u | limb) : 0u;
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
                    const u32 limb = b_limb(held);
                    if (limb != NONE) {
                        load(KIND_B, limb, held % UB);
                        held = NONE;
                        progress = true;
                    }
                } else {
                    bool claimed = false;
                    if (b_left && a_left) {
                        // A queue a_window limbs ahead: prefer a published B tile
                        const u32 peek = ld_relaxed(&a.ctl[1]);
                        if (peek >= totalB) b_left = false;
                        else if (ld_relaxed(&a.ctl[0]) / UA >= peek / UB + a.a_window && b_limb(peek) != NONE)
                            claim_b(claimed);
                    }
                    if (!claimed && a_left) {
                        const u32 t = atomicAdd(&a.ctl[0], 1u);
                        if (t < totalA) {
                            load(KIND_A, t / UA, t % UA);
                            claimed = true;
                        } else {
                            a_left = false;
                        }
                    }
                    if (!claimed && b_left) claim_b(claimed);
                    if (claimed) progress = true;
                    if (!a_left && !b_left && held == NONE) {
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
        if (atomicAdd(&a.ctl[2], 1u) == gridDim.x - 1) {
            for (u32 i = 0; i < 2 * a.limbs + 4; ++i) a.ctl[i] = 0u;
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
            // column pass: twiddles Psi[0, R1) staged with the tile
            if constexpr (FWD)
                compute_tile<P1, F::LOGC_COL, KMAX, false, true, 1, false, true, 0, true, NT, NoHook, true>(
                    sm, pr, buf_tw(b), nullptr, nullptr, 0u, 0u, tid);
            else
                compute_tile<P1, F::LOGC_COL, KMAX, false, false, X_B, true, true, 0, true, NT, NoHook, true>(
                    sm, pr, buf_tw(b), nullptr, nullptr, 0u, 0u, tid);
        } else {
            const FusedJobT<W>& J = a.job[MAXJ > 1 ? buf_desc(b)->job : 0u];
            const TwT* tw = J.tw + (size_t)pi * J.tw_len;
            const TwT* ota = J.ota ? J.ota + (size_t)pi * F::R2 : nullptr;
            const TwT* otb = J.otb ? J.otb + (size_t)pi * ((size_t)P2 << P1) : nullptr;
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
                if constexpr (FWD)
                    compute_tile<P2, LOGC_R, KMAX, true, true, X_B, true, false, OTS, false, NT, NoHook, true, false, W,
                                 STAGE, F::ROW_WARPX>(sm, pr, tw0, nullptr, nullptr, tile * F::CR, (u32)P1, tid,
                                                      NoHook(), htw, hw, ha);
                else
                    compute_tile<P2, LOGC_R, KMAX, true, false, 1, false, false, OTS, false, NT, NoHook, true, false, W,
                                 STAGE, F::ROW_WARPX>(sm, pr, tw0, nullptr, nullptr, tile * F::CR, (u32)P1, tid,
                                                      NoHook(), htw, hw, ha);
                ++rt;
            } else {
                if constexpr (FWD)
                    compute_tile<P2, LOGC_R, KMAX, true, true, X_B, true, false, OTS, false, NT, NoHook, true>(
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

// Uneven batches in one persistent launch: jobs of different sizes N and
// directions (the transforms of RNS polynomials at the different levels of an
// HE computation; Sec. V / VI-A batch the limbs of equal transforms).
//
// The jobs of a launch fall into groups of one size class (N = 2^13 .. 2^17,
// each with the default geometry of its size) and one direction.  Each group
// runs the two-phase protocol of the fused kernel (ntt_fused.cuh) on its own
// work area: phase-0 tiles never wait, a phase-1 tile waits for every phase-0
// tile of its limb, limbs are published in completion order.  The grid
// works through the groups in order: every CTA starts in group 0 and, once
// that group has no ticket left to claim, moves on to the next group that
// has, so at any time the SMs run the tile routines of one group (two at its
// end), which keeps them in the instruction caches, and the groups' tails
// overlap so that every CTA stays busy until all groups are done.  A unit descriptor
// carries the group, and the compute threads run the tile routine of its
// size class and direction.
//
// The per-job tensor maps live in a device array; the jobs' tables and the
// groups are kernel parameters (up to MIX_MAX_JOBS jobs per launch).
//
// Deadlock freedom: within a group the fused kernel's argument holds (a held
// ticket of phase 1 waits only for phase-0 tiles of that group, all claimed by
// CTAs that compute them); a CTA that holds a ticket stays in its group, and a
// CTA leaves a group only when that group has no ticket left to claim.
#pragma once
#include <type_traits>

#include "ntt_fused.cuh"

namespace ntt {

constexpr int MIX_MAX_GROUPS = 10;          // 5 size classes x 2 directions
constexpr int MIX_NT = 256;                 // compute threads
constexpr int MIX_FIRST_N = 13;             // size class c is N = 2^(13 + c)

// Geometry of size class c in a mixed launch: the default split and row tile
// of its size (geometry 0 of kGeometryTable).
template <int C>
struct MixGeom;
template <> struct MixGeom<0> { static constexpr int P1 = 6, P2 = 7, LOGC_R = 5; };   // N = 2^13
template <> struct MixGeom<1> { static constexpr int P1 = 7, P2 = 7, LOGC_R = 5; };   // N = 2^14
template <> struct MixGeom<2> { static constexpr int P1 = 7, P2 = 8, LOGC_R = 4; };   // N = 2^15
template <> struct MixGeom<3> { static constexpr int P1 = 8, P2 = 8, LOGC_R = 4; };   // N = 2^16
template <> struct MixGeom<4> { static constexpr int P1 = 8, P2 = 9, LOGC_R = 3; };   // N = 2^17
constexpr int MIX_CLASSES = 5;

template <int C, int KMAX, int OTS>
using MixCfg = FusedCfg<MixGeom<C>::P1, MixGeom<C>::P2, MixGeom<C>::LOGC_R, KMAX, u64, OTS>;

// Shared-memory layout of a mixed launch: the largest tile buffer and
// staged-twiddle buffer of the classes, two tile buffers when any class
// stages its row twiddles (else three).
template <int KMAX, int OTS>
struct MixLayout {
    template <int C>
    using Cf = MixCfg<C, KMAX, OTS>;
    static constexpr size_t mx(size_t a, size_t b) { return a > b ? a : b; }
    static constexpr int TILE = (int)mx(mx(mx(Cf<0>::TILE, Cf<1>::TILE), mx(Cf<2>::TILE, Cf<3>::TILE)), Cf<4>::TILE);
    static constexpr int R1 = 256;                     // largest column pass (2^8 rows)
    static constexpr size_t TW_OFF = (size_t)TILE * sizeof(u64);
    static constexpr size_t PR_OFF = TW_OFF + (size_t)R1 * sizeof(Tw);
    static constexpr size_t DESC_OFF = PR_OFF + sizeof(PrimeDev);
    static constexpr size_t BUF = (DESC_OFF + 32 + 1023) / 1024 * 1024;
    static constexpr bool ANY_STAGE = Cf<0>::STAGE || Cf<1>::STAGE || Cf<2>::STAGE || Cf<3>::STAGE || Cf<4>::STAGE;
    static constexpr size_t HTW_BYTES =
        mx(mx(mx(Cf<0>::HTW_BYTES, Cf<1>::HTW_BYTES), mx(Cf<2>::HTW_BYTES, Cf<3>::HTW_BYTES)), Cf<4>::HTW_BYTES);
    static constexpr int NBUF = ANY_STAGE ? 2 : 3;
    static constexpr size_t HTW_OFF = NBUF * BUF;
    static constexpr size_t SMEM = NBUF * BUF + HTW_BYTES + 1024;
    static constexpr int THREADS = MIX_NT + 32;
};

constexpr int MIX_MAX_JOBS = 128;           // jobs per mixed launch

// Tensor maps of one job of a mixed launch (device array, written by the
// host before the launch; the TMA unit reads them there).
struct __align__(128) MixJob {
    CUtensorMap mapC;            // column view of the job's data
    CUtensorMap mapR;            // row view
};

// The rest of a job, in the kernel parameters (constant cache: the
// producer's per-tile lookups stay off global memory).
struct MixJobInfo {
    const PrimeDev* primes;      // [L]
    const Tw* tw;                // [L][tw_len]
    const Tw* ota;               // OT factors of the job's direction
    const Tw* otb;
    u32 tw_len;
    u32 L;                       // primes per polynomial (local limb l uses prime l % L)
    u32 limb0;                   // first limb of the job in its group's numbering
    u32 reserved;
};

struct MixGroup {
    u32 cls;                     // size class (N = 2^(13 + cls))
    u32 fwd;                     // 1: forward transforms, 0: inverse
    u32 job0, njobs;             // the group's jobs are jobs [job0, job0 + njobs)
    u32 limbs;                   // limbs of all its jobs
    u32 ctl;                     // first word of the group's work area
};

struct MixParams {
    MixJobInfo info[MIX_MAX_JOBS];
    MixGroup group[MIX_MAX_GROUPS];
    const MixJob* jobs;
    u32* ctl;                    // work areas of the groups, then one word: CTAs finished
    u32* status;                 // persistent error word
    u32 ngroups;
    u32 ctl_words;               // all work-area words (zeroed by the last CTA)
    u32 max_polls;
    u32 reserved;
};

// Work-area words of a group of `limbs` limbs (the fused kernel's layout for
// two phases).
__host__ __device__ constexpr size_t mix_group_words(size_t limbs) { return fused_ctl_words(2, limbs); }

__device__ __forceinline__ void fence_tensormap(const CUtensorMap* m)
{
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"((uint64_t)m) : "memory");
}

template <int KMAX, int OTS>
__global__ void __launch_bounds__(MixLayout<KMAX, OTS>::THREADS, 2)
ntt_mixed_kernel(const __grid_constant__ MixParams a)
{
    using LY = MixLayout<KMAX, OTS>;
    constexpr int NT = MIX_NT;
    constexpr int NBUF = LY::NBUF;
    constexpr u32 NONE = 0xFFFFFFFFu;

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    auto buf_tile = [&](int b) { return reinterpret_cast<u64*>(smem_raw + b * LY::BUF); };
    auto buf_tw = [&](int b) { return reinterpret_cast<Tw*>(smem_raw + b * LY::BUF + LY::TW_OFF); };
    auto buf_pr = [&](int b) { return reinterpret_cast<PrimeDev*>(smem_raw + b * LY::BUF + LY::PR_OFF); };
    auto buf_desc = [&](int b) { return reinterpret_cast<volatile UnitDesc*>(smem_raw + b * LY::BUF + LY::DESC_OFF); };
    Tw* const htw = reinterpret_cast<Tw*>(smem_raw + LY::HTW_OFF);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + LY::HTW_OFF + LY::HTW_BYTES);
    uint64_t* empty = full + NBUF;
    uint64_t* htw_full = empty + NBUF;
    uint64_t* htw_empty = htw_full + 1;

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

    // phase 0 of a forward group is its column pass, of an inverse group its row pass
    auto is_col = [](u32 fwd, u32 kind) { return fwd ? kind == 0u : kind == 1u; };
    if (tid >= (u32)NT) {
        if (tid != (u32)NT) return;
        // =================================================== producer ====
        u32 issued = 0, stored = 0;
        u32 q0 = 0, q1 = 0, q2 = 0, qn = 0;      // committed stores not yet published: group << 28 | limb, +1
        u32 left = 0;                             // 2 bits per group: phases that may still have tickets
        for (u32 g = 0; g < a.ngroups; ++g) left |= 3u << (2 * g);
        // every CTA takes work from group 0 first and then from the groups in
        // order, so that the SMs run one group's tile routines at a time (the
        // groups' routines together exceed the instruction caches)
        u32 g = 0;
        bool stopped = false, failed = false;
        u32 held = NONE, held_g = 0;
        u32 idle = 0;
        u32 hq[NBUF > 1 ? NBUF : 1] = {};
        u32 hq_head = 0, hq_tail = 0, fills = 0;

        // the jobs' tensor maps are in global memory (written before the launch)
        for (u32 gg = 0; gg < a.ngroups; ++gg)
            for (u32 j = a.group[gg].job0; j < a.group[gg].job0 + a.group[gg].njobs; ++j) {
                fence_tensormap(&a.jobs[j].mapC);
                fence_tensormap(&a.jobs[j].mapR);
                prefetch_tensormap(&a.jobs[j].mapC);
                prefetch_tensormap(&a.jobs[j].mapR);
            }
        auto gctl = [&](u32 gg) { return a.ctl + a.group[gg].ctl; };
        auto units = [&](u32 gg, u32 p) -> u32 {
            const u32 c = a.group[gg].cls, n = MIX_FIRST_N + c;
            // column tiles: 2^(n - p1) / 16 per limb; row tiles: 2^p1 / CR
            u32 p1, lcr;
            switch (c) {
            case 0: p1 = MixGeom<0>::P1; lcr = MixGeom<0>::LOGC_R; break;
            case 1: p1 = MixGeom<1>::P1; lcr = MixGeom<1>::LOGC_R; break;
            case 2: p1 = MixGeom<2>::P1; lcr = MixGeom<2>::LOGC_R; break;
            case 3: p1 = MixGeom<3>::P1; lcr = MixGeom<3>::LOGC_R; break;
            default: p1 = MixGeom<4>::P1; lcr = MixGeom<4>::LOGC_R; break;
            }
            return is_col(a.group[gg].fwd, p) ? (1u << (n - p1)) >> 4 : (1u << p1) >> lcr;
        };
        auto job_of = [&](u32 gg, u32 limb) -> u32 {
            u32 lo = a.group[gg].job0, hi = lo + a.group[gg].njobs;
            while (hi - lo > 1) {
                const u32 mid = (lo + hi) >> 1;
                if (a.info[mid].limb0 <= limb) lo = mid;
                else hi = mid;
            }
            return lo;
        };
        auto pub_limb = [&](u32 gg, u32 i) -> u32 {
            const u32 limbs = a.group[gg].limbs;
            const u32 v = ld_acquire(gctl(gg) + 4 + limbs + i);
            return v ? v - 1u : NONE;
        };
        auto publish_entry = [&](u32 e) {
            if (e) {
                const u32 gg = (e >> 28) - 1u, limb = e & 0x0FFFFFFFu;
                u32* c = gctl(gg);
                fence_proxy_async_global();
                if (atom_acq_rel_add(&c[4 + limb], 1u) == units(gg, 0) - 1u) {
                    const u32 pos = atomicAdd(&c[2], 1u);
                    st_release(&c[4 + a.group[gg].limbs + pos], limb + 1u);
                }
            }
        };
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

        // class-specific steps of the producer
        auto do_fill = [&](auto cls_tag, const volatile UnitDesc* d) {
            constexpr int C = decltype(cls_tag)::value;
            using F = MixCfg<C, KMAX, OTS>;
            using RS = typename F::RS;
            constexpr int P1 = MixGeom<C>::P1, P2 = MixGeom<C>::P2;
            if constexpr (F::STAGE) {
                const MixJobInfo& J = a.info[d->job];
                const u32 pi = d->prime, u0 = d->tile * (u32)F::CR;
                const bool fwd = a.group[d->limb >> 28].fwd != 0;   // group in the high bits (see load)
                const Tw* base = J.tw + (size_t)pi * J.tw_len;
                mbar_arrive_expect_tx(htw_full, (u32)RS::NH * (u32)sizeof(Tw));
#pragma unroll
                for (int sl = RS::SSB; sl < P2 - OTS; ++sl) {
                    const u32 st = fwd ? (1u << (P1 + sl)) + (u0 << sl) : (2u << (P1 + sl)) - ((u0 + (u32)F::CR) << sl);
                    bulk_load(htw + F::CR * ((1 << sl) - (1 << RS::SSB)), base + st, ((u32)F::CR << sl) * (u32)sizeof(Tw),
                              htw_full);
                }
                if constexpr (OTS > 0) {
                    bulk_load(htw + RS::A_OFF, J.ota + (size_t)pi * F::R2 + (1u << (P2 - OTS)),
                              (u32)RS::NA * (u32)sizeof(Tw), htw_full);
#pragma unroll
                    for (int i = 0; i < OTS; ++i)
                        bulk_load(htw + RS::B_OFF + i * F::CR,
                                  J.otb + (size_t)pi * ((size_t)P2 << P1) + ((size_t)(P2 - OTS + i) << P1) + u0,
                                  (u32)F::CR * (u32)sizeof(Tw), htw_full);
                }
            }
        };
        auto fill_htw = [&]() -> bool {
            if constexpr (LY::ANY_STAGE) {
                if (hq_head == hq_tail) return false;
                if (fills && !mbar_test(htw_empty, (fills - 1) & 1u)) return false;
                const volatile UnitDesc* d = buf_desc((int)(hq[hq_head % NBUF] % NBUF));
                switch (a.group[d->limb >> 28].cls) {
                case 0: do_fill(std::integral_constant<int, 0>(), d); break;
                case 1: do_fill(std::integral_constant<int, 1>(), d); break;
                case 2: do_fill(std::integral_constant<int, 2>(), d); break;
                case 3: do_fill(std::integral_constant<int, 3>(), d); break;
                default: do_fill(std::integral_constant<int, 4>(), d); break;
                }
                ++hq_head;
                ++fills;
                return true;
            } else {
                return false;
            }
        };
        // load a unit (group gg, phase kind, group limb, tile); the descriptor's
        // limb field carries the group in its top 4 bits
        auto do_load = [&](auto cls_tag, u32 gg, u32 kind, u32 limb, u32 tile) {
            constexpr int C = decltype(cls_tag)::value;
            using F = MixCfg<C, KMAX, OTS>;
            using RS = typename F::RS;
            constexpr int P1 = MixGeom<C>::P1;
            const int b = (int)(issued % NBUF);
            const u32 j = job_of(gg, limb);
            const MixJobInfo& J = a.info[j];
            const MixJob& M = a.jobs[j];
            const u32 local = limb - J.limb0, pi = local % J.L;
            const bool fwd = a.group[gg].fwd != 0;
            volatile UnitDesc* d = buf_desc(b);
            d->kind = kind;
            d->limb = (gg << 28) | limb;
            d->tile = tile;
            d->prime = pi;
            d->job = j;
            d->local = local;
            bulk_wait_read<NBUF == 2 ? 0 : 1>();   // the buffer's previous store has read it
            if (kind > 0) fence_proxy_async_global();
            u64* dst = buf_tile(b);
            if (is_col(fwd, kind)) {
                mbar_arrive_expect_tx(&full[b], F::TILE_C * 8u + F::R1 * (u32)sizeof(Tw) + (u32)sizeof(PrimeDev));
                tma_load_2d(dst, &M.mapC, (int)(tile * F::COLW), (int)(local * F::R1), &full[b]);
                bulk_load(buf_tw(b), J.tw + (size_t)pi * J.tw_len, F::R1 * (u32)sizeof(Tw), &full[b]);
            } else {
                mbar_arrive_expect_tx(&full[b], F::TILE_R * 8u + (u32)sizeof(PrimeDev) + (u32)RS::N0 * (u32)sizeof(Tw));
                tma_load_2d(dst, &M.mapR, 0, (int)(local * (F::R1 * F::R2 / F::COLW) + tile * (F::TILE_R / F::COLW)),
                            &full[b]);
                const Tw* base = J.tw + (size_t)pi * J.tw_len;
                const u32 u0 = tile * (u32)F::CR;
                auto run_start = [&](int sl) -> u32 {
                    return fwd ? (1u << (P1 + sl)) + (u0 << sl) : (2u << (P1 + sl)) - ((u0 + (u32)F::CR) << sl);
                };
                if constexpr (F::STAGE == 1) {
#pragma unroll
                    for (int sl = 0; sl < RS::KR0; ++sl)
                        bulk_load(buf_tw(b) + F::CR * ((1 << sl) - 1), base + run_start(sl),
                                  ((u32)F::CR << sl) * (u32)sizeof(Tw), &full[b]);
                }
                if constexpr (F::STAGE) {
                    hq[hq_tail++ % NBUF] = issued;
                } else {
#pragma unroll
                    for (int sl = 0; sl < MixGeom<C>::P2 - OTS; ++sl)
                        bulk_prefetch_l2(base + run_start(sl), ((u32)F::CR << sl) * (u32)sizeof(Tw));
                }
            }
            bulk_load(buf_pr(b), J.primes + pi, (u32)sizeof(PrimeDev), &full[b]);
            ++issued;
        };
        auto load = [&](u32 gg, u32 kind, u32 limb, u32 tile) {
            switch (a.group[gg].cls) {
            case 0: do_load(std::integral_constant<int, 0>(), gg, kind, limb, tile); break;
            case 1: do_load(std::integral_constant<int, 1>(), gg, kind, limb, tile); break;
            case 2: do_load(std::integral_constant<int, 2>(), gg, kind, limb, tile); break;
            case 3: do_load(std::integral_constant<int, 3>(), gg, kind, limb, tile); break;
            default: do_load(std::integral_constant<int, 4>(), gg, kind, limb, tile); break;
            }
        };
        auto do_store = [&](auto cls_tag, int b, const volatile UnitDesc* d) {
            constexpr int C = decltype(cls_tag)::value;
            using F = MixCfg<C, KMAX, OTS>;
            const u32 gg = d->limb >> 28;
            const MixJob& M = a.jobs[d->job];
            const u64* src = buf_tile(b);
            if (is_col(a.group[gg].fwd, d->kind))
                tma_store_2d(&M.mapC, (int)(d->tile * F::COLW), (int)(d->local * F::R1), src);
            else
                tma_store_2d(&M.mapR, 0, (int)(d->local * (F::R1 * F::R2 / F::COLW) + d->tile * (F::TILE_R / F::COLW)),
                             src);
        };
        // claim in group gg (the fused kernel's rules for two phases); false
        // when the group has no ticket left
        auto claim = [&](u32 gg) -> bool {
            u32* c = gctl(gg);
            const u32 limbs = a.group[gg].limbs;
            const u32 sh = 2 * gg;
            if ((left >> sh) & 2u) {
                const u32 tot = limbs * units(gg, 1);
                const u32 t = ld_relaxed(&c[1]);
                if (t >= tot) {
                    left &= ~(2u << sh);
                } else {
                    const u32 limb = pub_limb(gg, t / units(gg, 1));
                    if (limb != NONE && atomicCAS(&c[1], t, t + 1u) == t) {
                        load(gg, 1, limb, t % units(gg, 1));
                        return true;
                    }
                }
            }
            if ((left >> sh) & 1u) {
                const u32 t = atomicAdd(&c[0], 1u);
                if (t < limbs * units(gg, 0)) {
                    load(gg, 0, t / units(gg, 0), t % units(gg, 0));
                    return true;
                }
                left &= ~(1u << sh);
            }
            if (((left >> sh) & 3u) == 2u) {
                const u32 t = atomicAdd(&c[1], 1u);
                if (t < limbs * units(gg, 1)) {
                    const u32 limb = pub_limb(gg, t / units(gg, 1));
                    if (limb != NONE) {
                        load(gg, 1, limb, t % units(gg, 1));
                    } else {
                        held = t;
                        held_g = gg;
                    }
                    return true;
                }
                left &= ~(2u << sh);
            }
            return false;
        };

        for (;;) {
            bool progress = fill_htw();
            while (stored < issued && mbar_test(&empty[stored % NBUF], (stored / NBUF) & 1u)) {
                const int b = (int)(stored % NBUF);
                const volatile UnitDesc* d = buf_desc(b);
                const u32 gg = d->limb >> 28, limb = d->limb & 0x0FFFFFFFu, kind = d->kind;
                switch (a.group[gg].cls) {
                case 0: do_store(std::integral_constant<int, 0>(), b, d); break;
                case 1: do_store(std::integral_constant<int, 1>(), b, d); break;
                case 2: do_store(std::integral_constant<int, 2>(), b, d); break;
                case 3: do_store(std::integral_constant<int, 3>(), b, d); break;
                default: do_store(std::integral_constant<int, 4>(), b, d); break;
                }
                bulk_commit();
                const u32 e = kind == 0u ? ((gg + 1u) << 28) | limb : 0u;
                if (qn == 0) q0 = e;
                else if (qn == 1) q1 = e;
                else q2 = e;
                ++qn;
                ++stored;
                publish_older();
                progress = true;
            }
            if (stopped) {
                if (stored + 1 == issued) break;
            } else if (issued - stored < 2u) {
                if (held != NONE) {
                    const u32 limb = pub_limb(held_g, held / units(held_g, 1));
                    if (limb != NONE) {
                        load(held_g, 1, limb, held % units(held_g, 1));
                        held = NONE;
                        progress = true;
                    }
                } else {
                    // this group, else the next one with tickets left
                    bool claimed = false;
                    for (u32 k = 0; k < a.ngroups && !claimed; ++k) {
                        if ((left >> (2 * g)) & 3u) claimed = claim(g);
                        if (!claimed) g = g + 1 < a.ngroups ? g + 1 : 0;
                    }
                    if (claimed) progress = true;
                    if (left == 0 && held == NONE) {
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
            publish_all();
            if (++idle > a.max_polls) {
                failed = true;
                break;
            }
            if (stored < issued && (held == NONE || issued - stored >= 2u) && hq_head == hq_tail)
                mbar_try_wait(&empty[stored % NBUF], (stored / NBUF) & 1u);
            else
                __nanosleep(held != NONE ? 256 : 64);
        }
        publish_all();
        for (u32 k = issued > (u32)NBUF ? issued - (u32)NBUF : 0u; k < issued; ++k)
            mbar_wait(&full[k % NBUF], (k / NBUF) & 1u, a.max_polls);
        if (LY::ANY_STAGE && fills) mbar_wait(htw_full, (fills - 1) & 1u, a.max_polls);
        if (failed) {
            atomicOr(a.status, held != NONE ? STATUS_DEP_TIMEOUT : STATUS_TMA_TIMEOUT);
            if (!stopped && issued - stored < (u32)NBUF) {
                const int b = (int)(issued % NBUF);
                buf_desc(b)->kind = KIND_STOP;
                mbar_arrive(&full[b]);
            }
        }
        __threadfence();
        if (atomicAdd(&a.ctl[a.ctl_words - 1], 1u) == gridDim.x - 1) {
            for (u32 i = 0; i < a.ctl_words; ++i) a.ctl[i] = 0u;
            __threadfence();
        }
        return;
    }

    // ===================================================== compute ======
    u32 rt = 0;
    bool htw_lost = false;
    auto run_unit = [&](auto cls_tag, int b, u32 fwd, u32 kind) {
        constexpr int C = decltype(cls_tag)::value;
        using F = MixCfg<C, KMAX, OTS>;
        constexpr int P1 = MixGeom<C>::P1, P2 = MixGeom<C>::P2, LOGC_R = MixGeom<C>::LOGC_R;
        constexpr int X_RF = ct_range_after(1, P1), X_CI = gs_range_after(1, P2);
        constexpr bool WARPX = rows_stay_in_warp<P2, LOGC_R, KMAX, NT>();
        const u32 tile = buf_desc(b)->tile, pi = buf_desc(b)->prime;
        u64* sm = buf_tile(b);
        const PrimeDev& pr = *buf_pr(b);
        if (is_col(fwd, kind)) {
            if (fwd)
                compute_tile<P1, 4, KMAX, false, true, 1, false, true, 0, true, NT, NoHook, true>(
                    sm, pr, buf_tw(b), nullptr, nullptr, 0u, 0u, tid);
            else
                compute_tile<P1, 4, KMAX, false, false, X_CI, true, true, 0, true, NT, NoHook, true>(
                    sm, pr, buf_tw(b), nullptr, nullptr, 0u, 0u, tid);
        } else if constexpr (F::STAGE) {
            const u32 ph = rt & 1u;
            auto hw = [&]() {
                if (!mbar_wait(htw_full, ph, a.max_polls)) htw_lost = true;
            };
            auto ha = [&]() { mbar_arrive(htw_empty); };
            const Tw* tw0 = F::STAGE == 1 ? buf_tw(b) : htw;
            if (fwd)
                compute_tile<P2, LOGC_R, KMAX, true, true, X_RF, true, false, OTS, false, NT, NoHook, true, false, u64,
                             F::STAGE, WARPX>(sm, pr, tw0, nullptr, nullptr, tile * F::CR, (u32)P1, tid, NoHook(), htw,
                                              hw, ha);
            else
                compute_tile<P2, LOGC_R, KMAX, true, false, 1, false, false, OTS, false, NT, NoHook, true, false, u64,
                             F::STAGE, WARPX>(sm, pr, tw0, nullptr, nullptr, tile * F::CR, (u32)P1, tid, NoHook(), htw,
                                              hw, ha);
            ++rt;
        } else {
            const MixJobInfo& J = a.info[buf_desc(b)->job];
            const Tw* tw = J.tw + (size_t)pi * J.tw_len;
            const Tw* ota = J.ota ? J.ota + (size_t)pi * F::R2 : nullptr;
            const Tw* otb = J.otb ? J.otb + (size_t)pi * ((size_t)P2 << P1) : nullptr;
            if (fwd)
                compute_tile<P2, LOGC_R, KMAX, true, true, X_RF, true, false, OTS, false, NT, NoHook, true>(
                    sm, pr, tw, ota, otb, tile * F::CR, (u32)P1, tid);
            else
                compute_tile<P2, LOGC_R, KMAX, true, false, 1, false, false, OTS, false, NT, NoHook, true, true>(
                    sm, pr, tw, ota, otb, tile * F::CR, (u32)P1, tid);
        }
    };
    for (u32 k = 0;; ++k) {
        const int b = (int)(k % NBUF);
        const bool got = mbar_wait(&full[b], (k / NBUF) & 1u, a.max_polls);
        if (compute_any<NT>(!got || htw_lost)) {
            if (tid == 0) atomicOr(a.status, STATUS_TMA_TIMEOUT);
            break;
        }
        const u32 kind = buf_desc(b)->kind;
        if (kind == KIND_STOP) break;
        const u32 gg = buf_desc(b)->limb >> 28;
        const u32 fwd = a.group[gg].fwd;
        switch (a.group[gg].cls) {
        case 0: run_unit(std::integral_constant<int, 0>(), b, fwd, kind); break;
        case 1: run_unit(std::integral_constant<int, 1>(), b, fwd, kind); break;
        case 2: run_unit(std::integral_constant<int, 2>(), b, fwd, kind); break;
        case 3: run_unit(std::integral_constant<int, 3>(), b, fwd, kind); break;
        default: run_unit(std::integral_constant<int, 4>(), b, fwd, kind); break;
        }
        fence_proxy_async_shared();
        mbar_arrive(&empty[b]);
    }
}

}  // namespace ntt

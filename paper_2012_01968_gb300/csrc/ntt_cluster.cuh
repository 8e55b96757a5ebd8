// One limb of N = 2^10 .. 2^12 on a thread-block cluster: the latency path of
// small transforms (one or a few limbs), where a single CTA would run all
// n stages of a limb on one SM.
//
// The limb is viewed as an R1 x R2 matrix (R1 = 2^p1 rows, p1 = floor(n/2),
// R2 = 2^(n - p1) columns, word v R2 + c), transformed as two passes of the
// merged negacyclic transform (Algorithm 1 split into p1 column stages and
// n - p1 row stages, Sec. VI-C): the column pass is R2 independent R1-point
// sub-transforms (twiddles Psi[0, R1)), the row pass R1 independent R2-point
// sub-transforms (twiddles of row u: Psi[2^(p1+s) + (u << s) + j]).  The
// inverse runs the row pass first, then the column pass (Gentleman-Sande,
// Algorithm 2 order).
//
// A cluster of CS = N / 512 CTAs holds the limb in shared memory, 512 words
// per CTA: CTA k owns columns [k CC, (k+1) CC) for the column pass and rows
// [k CR, (k+1) CR) for the row pass.  Between the passes every CTA gathers
// its tile of the other pass from the cluster's shared memory (distributed
// shared memory loads, 16 bytes each), after a cluster barrier that makes
// the producing pass's writes visible.  Global memory is read once (tile,
// the column twiddles and the tile's row-twiddle runs, all issued before any
// compute) and written once.  Forward then inverse (MODE 2) keeps the
// forward's row tile in place for the inverse's row pass: two exchanges for
// the pair instead of four.
//
// Waits: the cluster barriers (every CTA of the cluster runs the same
// sequence and none exits early) and the block barriers of the tile
// routines; no polling.  A CTA leaves only after a last cluster barrier, so
// no CTA reads the shared memory of one that has exited.
#pragma once
#include "ntt_pass.cuh"

namespace ntt {

constexpr int CLUSTER_KMAX = 3;            // stages per thread per round
constexpr int CLUSTER_MIN_N = 10, CLUSTER_MAX_N = 12;
constexpr int CLUSTER_TILE_LOG = 9;        // 512 words per CTA

template <int NLOG>
struct ClusterCfg {
    static_assert(NLOG >= CLUSTER_MIN_N && NLOG <= CLUSTER_MAX_N, "cluster sizes");
    static constexpr int P1 = NLOG / 2, P2 = NLOG - P1;
    static constexpr int CSL = NLOG - CLUSTER_TILE_LOG;     // log2 of the cluster size
    static constexpr int CS = 1 << CSL;
    static constexpr int R1 = 1 << P1, R2 = 1 << P2;
    static constexpr int LOGC_C = P2 - CSL, LOGC_R = P1 - CSL;
    static constexpr int CC = 1 << LOGC_C;                  // columns per CTA
    static constexpr int CR = 1 << LOGC_R;                  // rows per CTA
    static constexpr int TILE = 1 << CLUSTER_TILE_LOG;
    static constexpr int TC = pass_threads(P1, LOGC_C, CLUSTER_KMAX);
    static constexpr int TR = pass_threads(P2, LOGC_R, CLUSTER_KMAX);
    static constexpr int NT = TC > TR ? TC : TR;
    static constexpr int NH = CR * (R2 - 1);                // row-twiddle runs of one tile, all row stages
    static_assert(CC >= 2 && CR >= 1 && TILE / 2 % NT == 0, "tile shape");
};

struct ClusterArgs {
    u64* data;               // [limbs][N]
    const PrimeDev* primes;  // [L]
    const Tw* tw;            // [L][N], slot order of the cluster's two passes
    u32 L;
    u32 limbs;
};

__device__ __forceinline__ u32 cluster_rank()
{
    u32 r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ u32 cluster_id_x()
{
    u32 r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
// every thread of every CTA of the cluster: the writes before it are visible
// to the reads after it, cluster-wide
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_sync()
{
    cluster_arrive();
    cluster_wait();
}
// shared-memory address of the same variable in CTA `rank` of the cluster
__device__ __forceinline__ u32 cluster_map(const void* p, u32 rank)
{
    u32 r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
                 : "=r"(r)
                 : "r"((u32)__cvta_generic_to_shared(p)), "r"(rank));
    return r;
}
__device__ __forceinline__ void ld_cluster_pair(u32 addr, u64& a, u64& b)
{
    asm volatile("ld.shared::cluster.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "r"(addr) : "memory");
}

// The row tile of CTA `rank` (rows [rank CR, +CR), word r R2 + c) from the
// column tiles of the cluster (CTA j holds columns [j CC, +CC), word v CC + cc).
template <class CF>
__device__ __forceinline__ void gather_rows(u64* rowbuf, const u64* colbuf, u32 rank, u32 tid)
{
    constexpr int PER = CF::TILE / 2 / CF::NT;
    u64 x[PER][2];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const u32 w = 2u * (tid + (u32)k * CF::NT);          // even word of the row tile
        const u32 r = w >> CF::P2, c = w & (CF::R2 - 1);
        const u32 j = c >> CF::LOGC_C, cc = c & (CF::CC - 1);
        const u32 src = (rank * CF::CR + r) * CF::CC + cc;
        ld_cluster_pair(cluster_map(colbuf + swz(src), j), x[k][0], x[k][1]);
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const u32 w = 2u * (tid + (u32)k * CF::NT);
        store_pair(rowbuf + swz(w), x[k][0], x[k][1]);
    }
}

// The column tile of CTA `rank` (columns [rank CC, +CC), word v CC + cc) from
// the row tiles of the cluster (CTA j holds rows [j CR, +CR)).
template <class CF>
__device__ __forceinline__ void gather_cols(u64* colbuf, const u64* rowbuf, u32 rank, u32 tid)
{
    constexpr int PER = CF::TILE / 2 / CF::NT;
    u64 x[PER][2];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const u32 w = 2u * (tid + (u32)k * CF::NT);          // even word of the column tile
        const u32 v = w >> CF::LOGC_C, cc = w & (CF::CC - 1);
        const u32 j = v >> CF::LOGC_R, r = v & (CF::CR - 1);
        const u32 src = r * CF::R2 + rank * CF::CC + cc;
        ld_cluster_pair(cluster_map(rowbuf + swz(src), j), x[k][0], x[k][1]);
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const u32 w = 2u * (tid + (u32)k * CF::NT);
        store_pair(colbuf + swz(w), x[k][0], x[k][1]);
    }
}

// The row-twiddle runs of the tile of rows [u0, u0 + CR), stage after stage
// (stage sl: CR << sl entries at offset CR (2^sl - 1)), the forward's
// ascending runs or the inverse's mirrored ones; every load is issued before
// the first store.
template <class CF, bool FWDDIR>
__device__ __forceinline__ void load_row_runs(Tw* dst, const Tw* tw, u32 u0, u32 tid)
{
    constexpr int K = (CF::NH + CF::NT - 1) / CF::NT;
    Tw t[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const u32 e = tid + (u32)k * CF::NT;
        if (e < (u32)CF::NH) {
            const u32 sl = 31u - (u32)__clz((int)(e / CF::CR + 1u));     // CR (2^sl - 1) <= e < CR (2^(sl+1) - 1)
            const u32 i = e - (u32)CF::CR * ((1u << sl) - 1u);
            const u32 src = FWDDIR ? (1u << (CF::P1 + sl)) + (u0 << sl) + i
                                   : (2u << (CF::P1 + sl)) - ((u0 + (u32)CF::CR) << sl) + i;
            t[k] = tw[src];
        }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const u32 e = tid + (u32)k * CF::NT;
        if (e < (u32)CF::NH) dst[e] = t[k];
    }
}

// MODE 0: forward; 1: inverse; 2: forward, then the inverse of its result.
template <int NLOG, int MODE>
__global__ void __launch_bounds__(ClusterCfg<NLOG>::NT) ntt_cluster_kernel(const ClusterArgs a)
{
    using CF = ClusterCfg<NLOG>;
    constexpr int NT = CF::NT, P1 = CF::P1, P2 = CF::P2, KM = CLUSTER_KMAX;
    constexpr int PER = CF::TILE / 2 / NT;
    constexpr bool DO_FWD = MODE != 1, DO_INV = MODE != 0;
    __shared__ __align__(16) u64 colbuf[CF::TILE];
    __shared__ __align__(16) u64 rowbuf[CF::TILE];
    __shared__ __align__(16) Tw twc[CF::R1];                    // Psi[0, R1): the column pass
    __shared__ __align__(16) Tw twf[DO_FWD ? CF::NH : 1];      // the forward row pass's runs
    __shared__ __align__(16) Tw twi[DO_INV ? CF::NH : 1];      // the inverse row pass's runs
    __shared__ __align__(16) PrimeDev prs;

    const u32 tid = threadIdx.x;
    const u32 rank = cluster_rank();
    const u32 limb = cluster_id_x();
    const u32 pi = limb % a.L;
    u64* const base = a.data + ((size_t)limb << NLOG);
    const Tw* const tw = a.tw + ((size_t)pi << NLOG);
    const u32 u0 = rank * CF::CR;                                // first row of this CTA's row tile

    // ---- every global read of the launch, issued before any compute -----
    if (tid == 0) prs = a.primes[pi];
    for (u32 i = tid; i < (u32)CF::R1; i += NT) twc[i] = tw[i];
    if constexpr (DO_FWD) load_row_runs<CF, true>(twf, tw, u0, tid);
    if constexpr (DO_INV) load_row_runs<CF, false>(twi, tw, u0, tid);
    {
        ulonglong2 v[PER];
        if constexpr (DO_FWD) {
            // column tile: R1 rows of CC words, row v at v R2 + rank CC
#pragma unroll
            for (int k = 0; k < PER; ++k) {
                const u32 w = 2u * (tid + (u32)k * NT), r = w >> CF::LOGC_C, cc = w & (CF::CC - 1);
                v[k] = *reinterpret_cast<const ulonglong2*>(base + (size_t)r * CF::R2 + rank * CF::CC + cc);
            }
#pragma unroll
            for (int k = 0; k < PER; ++k) store_pair(colbuf + swz(2u * (tid + (u32)k * NT)), v[k].x, v[k].y);
        } else {
            // row tile: CR whole rows, contiguous
            const ulonglong2* src = reinterpret_cast<const ulonglong2*>(base + (size_t)u0 * CF::R2);
#pragma unroll
            for (int k = 0; k < PER; ++k) v[k] = src[tid + (u32)k * NT];
#pragma unroll
            for (int k = 0; k < PER; ++k) store_pair(rowbuf + swz(2u * (tid + (u32)k * NT)), v[k].x, v[k].y);
        }
    }
    __syncthreads();

    if constexpr (DO_FWD) {
        compute_tile<P1, CF::LOGC_C, KM, false, true, 1, false, true, 0, true, NT>(colbuf, prs, twc, nullptr,
                                                                                  nullptr, 0u, 0u, tid);
        cluster_sync();                                 // every column tile computed
        gather_rows<CF>(rowbuf, colbuf, rank, tid);
        if constexpr (MODE == 0) cluster_arrive();      // this CTA has read the others' column tiles
        __syncthreads();
        constexpr int X_RF = ct_range_after(1, P1);
        compute_tile<P2, CF::LOGC_R, KM, true, true, X_RF, true, false, 0, false, NT, NoHook, false, false, u64, 2>(
            rowbuf, prs, twf, nullptr, nullptr, u0, (u32)P1, tid, NoHook(), twf);
    }
    if constexpr (DO_INV) {
        if constexpr (MODE == 2) __syncthreads();
        compute_tile<P2, CF::LOGC_R, KM, true, false, 1, false, false, 0, false, NT, NoHook, false, false, u64, 2>(
            rowbuf, prs, twi, nullptr, nullptr, u0, (u32)P1, tid, NoHook(), twi);
        // every row tile computed; with MODE 2 every CTA has also finished
        // reading the column tiles, which the gather now overwrites
        cluster_sync();
        gather_cols<CF>(colbuf, rowbuf, rank, tid);
        cluster_arrive();                               // this CTA has read the others' row tiles
        __syncthreads();
        constexpr int X_CI = gs_range_after(1, P2);
        compute_tile<P1, CF::LOGC_C, KM, false, false, X_CI, true, true, 0, true, NT>(colbuf, prs, twc, nullptr,
                                                                                     nullptr, 0u, 0u, tid);
    }
    __syncthreads();

    // ---- write back: the row tile (forward) or the column tile ------------
    if constexpr (MODE == 0) {
        ulonglong2* dst = reinterpret_cast<ulonglong2*>(base + (size_t)u0 * CF::R2);
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            u64 x0, x1;
            load_pair(rowbuf + swz(2u * (tid + (u32)k * NT)), x0, x1);
            dst[tid + (u32)k * NT] = make_ulonglong2(x0, x1);
        }
    } else {
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const u32 w = 2u * (tid + (u32)k * NT), r = w >> CF::LOGC_C, cc = w & (CF::CC - 1);
            u64 x0, x1;
            load_pair(colbuf + swz(w), x0, x1);
            *reinterpret_cast<ulonglong2*>(base + (size_t)r * CF::R2 + rank * CF::CC + cc) = make_ulonglong2(x0, x1);
        }
    }
    // no CTA leaves while another may still read its shared memory
    cluster_wait();
}

}  // namespace ntt

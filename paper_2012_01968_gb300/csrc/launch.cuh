// Host-side launch helpers for the pass kernels.
#pragma once
#include <cuda_runtime.h>

#include <mutex>

#include "ntt_fused.cuh"
#include "ntt_pass.cuh"
#include "plan.h"

namespace ntt {

constexpr u32 kMaxGridY = 65535;

// Launch `kern` with an optional L2 access-policy window (persisting hits on
// [base, base + bytes), streaming misses); a plain launch when bytes == 0.
template <class Kern, class Arg>
cudaError_t launch_windowed(Kern kern, dim3 grid, dim3 block, size_t smem, cudaStream_t s, const void* base,
                            size_t bytes, float hit, const Arg& arg)
{
    if (bytes == 0) {
        kern<<<grid, block, smem, s>>>(arg);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeAccessPolicyWindow;
    attr[0].val.accessPolicyWindow.base_ptr = const_cast<void*>(base);
    attr[0].val.accessPolicyWindow.num_bytes = bytes;
    attr[0].val.accessPolicyWindow.hitRatio = hit;
    attr[0].val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
    attr[0].val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, arg);
}

// What one pass launch needs, for either word size.
template <class W>
struct PassLaunch {
    W* data;
    u32 limbs, L, n;
    const typename WordTypes<W>::Prime* primes;
    const typename WordTypes<W>::Tw* tw;
    u32 tw_len;
    cudaStream_t stream;
    const void* l2_base = nullptr;   // L2 access-policy window (l2_bytes 0: none)
    size_t l2_bytes = 0;
    float l2_hit = 0.f;
};

template <int P, int LOGC, int KMAX, bool ROWS, bool FWD, int XIN, bool FINAL, bool HAS_S0, int OTS,
          bool TW_SMEM, class W, bool TBL_LAST = false>
cudaError_t launch_pass_w(const PassLaunch<W>& c, u32 s0, const typename WordTypes<W>::Tw* ota,
                          const typename WordTypes<W>::Tw* otb)
{
    auto kern = ntt_pass_kernel<P, LOGC, KMAX, ROWS, FWD, XIN, FINAL, HAS_S0, OTS, TW_SMEM, W, TBL_LAST>;
    constexpr size_t smem = pass_smem_bytes<P, LOGC, KMAX, ROWS, HAS_S0, TW_SMEM, OTS, W>();
    constexpr int T = pass_threads(P, LOGC, KMAX);
    if (smem > 48 * 1024) {
        static std::once_flag once;
        static cudaError_t attr_err = cudaSuccess;
        std::call_once(once, [&] {
            attr_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        });
        if (attr_err != cudaSuccess) return attr_err;
    }
    const u32 tiles = (1u << c.n) >> (P + LOGC);
    PassArgsT<W> a;
    a.data = c.data;
    a.primes = c.primes;
    a.tw = c.tw;
    a.ota = ota;
    a.otb = otb;
    a.prime_map = nullptr;
    a.tw_len = c.tw_len;
    a.n = c.n;
    a.s0 = s0;
    a.b = c.n - s0 - P;
    a.L = c.L;
    for (u32 off = 0; off < c.limbs; off += kMaxGridY) {
        const u32 cnt = c.limbs - off < kMaxGridY ? c.limbs - off : kMaxGridY;
        a.limb_offset = off;
        const cudaError_t e = launch_windowed(kern, dim3(tiles, cnt), dim3(T), smem, c.stream, c.l2_base,
                                              c.l2_bytes, c.l2_hit, a);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <int P, int LOGC, int KMAX, bool ROWS, bool FWD, int XIN, bool FINAL, bool HAS_S0, int OTS,
          bool TW_SMEM, bool TBL_LAST = false>
cudaError_t launch_pass(const LaunchCtx& c, u32 s0, const Tw* ota, const Tw* otb)
{
    const PassLaunch<u64> pl{c.data,   c.limbs,    c.L,        c.n,        c.primes,
                             c.tw,     c.tw_len,   c.stream,   c.l2_base,  c.l2_bytes, c.l2_hit};
    return launch_pass_w<P, LOGC, KMAX, ROWS, FWD, XIN, FINAL, HAS_S0, OTS, TW_SMEM, u64, TBL_LAST>(pl, s0, ota, otb);
}

// Single pass over all n stages (n <= 12): one CTA per limb, with the limb's
// whole table Psi[0, N) staged in shared memory beside the data (one batched
// copy before the first round instead of a global read in every stage).
template <int N_LOG>
cudaError_t launch_single_n(const LaunchCtx& c, bool fwd)
{
    if (fwd)
        return launch_pass<N_LOG, 0, KMAX_ALL, true, true, 1, true, true, 0, true>(c, 0, nullptr, nullptr);
    return launch_pass<N_LOG, 0, KMAX_ALL, true, false, 1, true, true, 0, true>(c, 0, nullptr, nullptr);
}

// Two passes: P1 column-like stages [0, P1), then P2 row-like stages.  The
// row passes take OTS on-the-fly stages with their factor tables; in table
// mode (OTS 0) they read the last stage's twiddles from the table in global
// memory instead (TBL_LAST), with the other stages' runs staged in shared
// memory as with one OT stage, so that they keep the shared-memory footprint
// of OT1 without its second product.
template <int P1, int P2, int LOGC_R, int KMAX_R, int OTS>
cudaError_t launch_two_pass_ots(const LaunchCtx& c, bool fwd)
{
    constexpr int LOGC_C = 4;
    constexpr int KMAX_C = KMAX_R;
    constexpr bool TBL_LAST = OTS == 0;
    constexpr int OTS_R = TBL_LAST ? 1 : OTS;
    cudaError_t e;
    if (fwd) {
        e = launch_pass<P1, LOGC_C, KMAX_C, false, true, 1, false, true, 0, true>(c, 0, nullptr, nullptr);
        if (e != cudaSuccess) return e;
        constexpr int X2 = ct_range_after(1, P1);
        return launch_pass<P2, LOGC_R, KMAX_R, true, true, X2, true, false, OTS_R, false, TBL_LAST>(c, P1, c.ota_f,
                                                                                                   c.otb_f);
    }
    e = launch_pass<P2, LOGC_R, KMAX_R, true, false, 1, false, false, OTS_R, false, TBL_LAST>(c, P1, c.ota_i, c.otb_i);
    if (e != cudaSuccess) return e;
    constexpr int X1 = gs_range_after(1, P2);
    return launch_pass<P1, LOGC_C, KMAX_C, false, false, X1, true, true, 0, true>(c, 0, nullptr, nullptr);
}

// 32-bit words (table twiddles, one launch per pass).  The column pass takes
// 32 columns per tile so that each row segment is a full 128-byte line.
template <int N_LOG>
cudaError_t launch_single_w32(const PassLaunch<u32>& c, bool fwd)
{
    if (fwd)
        return launch_pass_w<N_LOG, 0, KMAX_ALL, true, true, 1, true, true, 0, false, u32>(c, 0, nullptr, nullptr);
    return launch_pass_w<N_LOG, 0, KMAX_ALL, true, false, 1, true, true, 0, false, u32>(c, 0, nullptr, nullptr);
}

template <int P1, int P2, int LOGC_R, int KMAX_R>
cudaError_t launch_two_pass_w32(const PassLaunch<u32>& c, bool fwd)
{
    constexpr int LOGC_C = 5;
    cudaError_t e;
    if (fwd) {
        e = launch_pass_w<P1, LOGC_C, KMAX_R, false, true, 1, false, true, 0, true, u32>(c, 0, nullptr, nullptr);
        if (e != cudaSuccess) return e;
        constexpr int X2 = ct_range_after(1, P1);
        return launch_pass_w<P2, LOGC_R, KMAX_R, true, true, X2, true, false, 0, false, u32>(c, P1, nullptr, nullptr);
    }
    e = launch_pass_w<P2, LOGC_R, KMAX_R, true, false, 1, false, false, 0, false, u32>(c, P1, nullptr, nullptr);
    if (e != cudaSuccess) return e;
    constexpr int X1 = gs_range_after(1, P2);
    return launch_pass_w<P1, LOGC_C, KMAX_R, false, false, X1, true, true, 0, true, u32>(c, 0, nullptr, nullptr);
}

// 32-bit launchers by size (k_w32_single.cu: n <= 12, k_w32_two.cu: 13 <= n <= 17,
// one launch per pass; k_w32_fused.cu: 13 <= n <= 17, the fused kernel)
cudaError_t launch_w32_single(const PassLaunch<u32>& c, bool fwd);
cudaError_t launch_w32_two(const PassLaunch<u32>& c, bool fwd);
struct Fused32Launch;
cudaError_t launch_w32_fused(const Fused32Launch& c, bool fwd);

// host helpers for the fused launch (fused_host.cu)
cudaError_t encode_tile_maps(u64* data, u32 limbs, u32 n, int p1, int row_tile_words, CUtensorMap* mapC,
                             CUtensorMap* mapR);
cudaError_t encode_tile_maps32(u32* data, u32 limbs, u32 n, int p1, int row_tile_words, CUtensorMap* mapC,
                               CUtensorMap* mapR);
int device_sm_count();

// One persistent launch over all limbs of all jobs, both passes (CHAIN: the
// forward and then the inverse transform, four passes).
template <int P1, int P2, int LOGC_R, int KMAX, bool FWD, int OTS, int MAXJ, bool MULB = false, bool CHAIN = false>
cudaError_t launch_fused_dir(const JobsCtx& c)
{
    using F = FusedCfg<P1, P2, LOGC_R, KMAX, u64, OTS>;
    auto kern = ntt_fused_kernel<P1, P2, LOGC_R, KMAX, FWD, OTS, MAXJ, u64, MULB, CHAIN>;
    constexpr u32 NP = fused_phases<FWD, CHAIN>();
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    static int occ = 0;
    std::call_once(once, [&] {
        attr_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)F::SMEM);
        if (attr_err == cudaSuccess)
            attr_err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, F::THREADS, F::SMEM);
    });
    if (attr_err != cudaSuccess) return attr_err;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    if (c.njobs < 1 || c.njobs > (u32)MAXJ) return cudaErrorInvalidValue;
    FusedParams<MAXJ> a{};
    u64 limbs = 0;
    for (u32 j = 0; j < c.njobs; ++j) {
        const JobCtx& J = c.jobs[j];
        cudaError_t e = encode_tile_maps(J.data, J.limbs, c.n, P1, F::TILE_R, &a.mapC[j], &a.mapR[j]);
        if (e != cudaSuccess) return e;
        a.job[j].primes = J.primes;
        a.job[j].tw = J.tw;
        a.job[j].ota = FWD ? J.ota_f : J.ota_i;
        a.job[j].otb = FWD ? J.otb_f : J.otb_i;
        a.job[j].ota_inv = CHAIN ? J.ota_i : nullptr;
        a.job[j].otb_inv = CHAIN ? J.otb_i : nullptr;
        // a product operand is only taken by the MULB instantiation
        if ((J.mulb != nullptr) != MULB || (J.mulb && ((uintptr_t)J.mulb & 15u))) return cudaErrorInvalidValue;
        a.job[j].mulb = J.mulb;
        a.job[j].tw_len = J.tw_len;
        a.job[j].L = J.L;
        a.job[j].limb0 = (u32)limbs;
        limbs += J.limbs;
    }
    // limbs are numbered in 28 bits by the publication entries; the work area
    // must hold the launch's counters (fused_ctl_words)
    if (limbs == 0 || limbs >= (1ull << 28) || !c.work ||
        fused_work_words(c.work_limbs) < fused_ctl_words(NP, (size_t)limbs))
        return cudaErrorInvalidValue;
    constexpr u32 UC = F::R2 / 16, UR = F::R1 / F::CR;
    const u64 units = limbs * (UC + UR) * (CHAIN ? 2 : 1);
    const u64 per_sm = c.ctas_per_sm && c.ctas_per_sm < (u32)occ ? c.ctas_per_sm : (u32)occ;
    const u64 slots = (u64)device_sm_count() * per_sm;
    const u32 grid = (u32)(units < slots ? units : slots);
    a.ctl = c.work;
    a.status = c.status;
    a.njobs = c.njobs;
    a.limbs = (u32)limbs;
    a.max_polls = c.max_polls ? c.max_polls : 1u << 22;
    return launch_windowed(kern, dim3(grid), dim3(F::THREADS), F::SMEM, c.stream, c.l2_base, c.l2_bytes, c.l2_hit,
                           a);
}

template <int P1, int P2, int LOGC_R, int KMAX, int MAXJ>
cudaError_t launch_fused(const JobsCtx& c, bool fwd)
{
    if constexpr (MAXJ == 1) {
        // forward, then inverse, in one launch (one job)
        if (c.chain) {
            if (!fwd || c.njobs != 1 || c.jobs[0].mulb) return cudaErrorInvalidValue;
            switch (c.ots) {
            case 0: return launch_fused_dir<P1, P2, LOGC_R, KMAX, true, 0, 1, false, true>(c);
            case 1: return launch_fused_dir<P1, P2, LOGC_R, KMAX, true, 1, 1, false, true>(c);
            case 2: return launch_fused_dir<P1, P2, LOGC_R, KMAX, true, 2, 1, false, true>(c);
            default: return cudaErrorInvalidValue;
            }
        }
        // the inverse of an in-place negacyclic product (one job)
        if (!fwd && c.njobs == 1 && c.jobs[0].mulb) {
            switch (c.ots) {
            case 0: return launch_fused_dir<P1, P2, LOGC_R, KMAX, false, 0, 1, true>(c);
            case 1: return launch_fused_dir<P1, P2, LOGC_R, KMAX, false, 1, 1, true>(c);
            case 2: return launch_fused_dir<P1, P2, LOGC_R, KMAX, false, 2, 1, true>(c);
            default: return cudaErrorInvalidValue;
            }
        }
    }
    switch (c.ots) {
    case 0: return fwd ? launch_fused_dir<P1, P2, LOGC_R, KMAX, true, 0, MAXJ>(c)
                       : launch_fused_dir<P1, P2, LOGC_R, KMAX, false, 0, MAXJ>(c);
    case 1: return fwd ? launch_fused_dir<P1, P2, LOGC_R, KMAX, true, 1, MAXJ>(c)
                       : launch_fused_dir<P1, P2, LOGC_R, KMAX, false, 1, MAXJ>(c);
    case 2: return fwd ? launch_fused_dir<P1, P2, LOGC_R, KMAX, true, 2, MAXJ>(c)
                       : launch_fused_dir<P1, P2, LOGC_R, KMAX, false, 2, MAXJ>(c);
    default: return cudaErrorInvalidValue;
    }
}

// The fused kernel on 32-bit words (one job, table twiddles): what a launch needs.
struct Fused32Launch {
    u32* data;
    u32 limbs, L, n;
    const PrimeDev32* primes;
    const Tw32* tw;
    u32 tw_len;
    u32* status;
    u32* work;               // zero, fused_work_words(work_limbs) words
    u32 work_limbs;
    cudaStream_t stream;
    u32 ots;                 // last stages twiddled on the fly (0 or 1)
    const Tw32* ota;         // OT factors of this direction (ots > 0)
    const Tw32* otb;
};

template <int P1, int P2, int LOGC_R, int KMAX, bool FWD, int OTS>
cudaError_t launch_fused32_dir(const Fused32Launch& c)
{
    using F = FusedCfg<P1, P2, LOGC_R, KMAX, u32>;
    auto kern = ntt_fused_kernel<P1, P2, LOGC_R, KMAX, FWD, OTS, 1, u32>;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    static int occ = 0;
    std::call_once(once, [&] {
        attr_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)F::SMEM);
        if (attr_err == cudaSuccess)
            attr_err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, F::THREADS, F::SMEM);
    });
    if (attr_err != cudaSuccess) return attr_err;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    if (c.limbs == 0 || c.limbs > 0x7FFFFFFFu || !c.work || c.work_limbs < c.limbs) return cudaErrorInvalidValue;
    FusedParams<1, u32> a{};
    cudaError_t e = encode_tile_maps32(c.data, c.limbs, c.n, P1, F::TILE_R, &a.mapC[0], &a.mapR[0]);
    if (e != cudaSuccess) return e;
    a.job[0].primes = c.primes;
    a.job[0].tw = c.tw;
    a.job[0].ota = OTS ? c.ota : nullptr;
    a.job[0].otb = OTS ? c.otb : nullptr;
    a.job[0].tw_len = c.tw_len;
    a.job[0].L = c.L;
    a.job[0].limb0 = 0;
    constexpr u32 UC = F::R2 / F::COLW, UR = F::R1 / F::CR;
    const u64 units = (u64)c.limbs * (UC + UR);
    const u64 slots = (u64)device_sm_count() * (u64)occ;
    const u32 grid = (u32)(units < slots ? units : slots);
    a.ctl = c.work;
    a.status = c.status;
    a.njobs = 1;
    a.limbs = c.limbs;
    a.max_polls = 1u << 22;
    kern<<<grid, F::THREADS, F::SMEM, c.stream>>>(a);
    return cudaGetLastError();
}

template <int P1, int P2, int LOGC_R, int KMAX>
cudaError_t launch_fused32(const Fused32Launch& c, bool fwd)
{
    if (c.ots == 0)
        return fwd ? launch_fused32_dir<P1, P2, LOGC_R, KMAX, true, 0>(c)
                   : launch_fused32_dir<P1, P2, LOGC_R, KMAX, false, 0>(c);
    if (c.ots == 1)
        return fwd ? launch_fused32_dir<P1, P2, LOGC_R, KMAX, true, 1>(c)
                   : launch_fused32_dir<P1, P2, LOGC_R, KMAX, false, 1>(c);
    return cudaErrorInvalidValue;
}

// A single call: one launch per pass, or the fused kernel with one job.
template <int P1, int P2, int LOGC_R, int KMAX_R>
cudaError_t launch_two_pass(const LaunchCtx& c, bool fwd)
{
    if (c.separate_passes) {
        switch (c.ots) {
        case 0: return launch_two_pass_ots<P1, P2, LOGC_R, KMAX_R, 0>(c, fwd);
        case 1: return launch_two_pass_ots<P1, P2, LOGC_R, KMAX_R, 1>(c, fwd);
        case 2: return launch_two_pass_ots<P1, P2, LOGC_R, KMAX_R, 2>(c, fwd);
        default: return cudaErrorInvalidValue;
        }
    }
    const JobCtx job{c.data, c.limbs, c.L, c.primes, c.tw, c.tw_len, c.ota_f, c.otb_f, c.ota_i, c.otb_i, c.mulb};
    JobsCtx jc{&job,   1u,         c.n,      c.ots,        c.status,  c.work,   c.work_limbs,
               c.stream, c.max_polls, c.geom, c.l2_base, c.l2_bytes, c.l2_hit};
    jc.chain = c.chain;
    jc.ctas_per_sm = c.ctas_per_sm;
    return launch_fused<P1, P2, LOGC_R, KMAX_R, 1>(jc, fwd);
}

// Several jobs of one size in one fused launch.
template <int P1, int P2, int LOGC_R, int KMAX_R>
cudaError_t launch_jobs(const JobsCtx& c, bool fwd)
{
    return launch_fused<P1, P2, LOGC_R, KMAX_R, FUSED_MAX_JOBS>(c, fwd);
}

}  // namespace ntt

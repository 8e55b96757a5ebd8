// Host-side launch helpers for the pass kernels.
#pragma once
#include <cuda_runtime.h>

#include <mutex>

#include "ntt_fused.cuh"
#include "ntt_pass.cuh"
#include "plan.h"

namespace ntt {

constexpr u32 kMaxGridY = 65535;

template <int P, int LOGC, int KMAX, bool ROWS, bool FWD, int XIN, bool FINAL, bool HAS_S0, int OTS,
          bool TW_SMEM>
cudaError_t launch_pass(const LaunchCtx& c, u32 s0, const Tw* ota, const Tw* otb)
{
    auto kern = ntt_pass_kernel<P, LOGC, KMAX, ROWS, FWD, XIN, FINAL, HAS_S0, OTS, TW_SMEM>;
    constexpr size_t smem = pass_smem_bytes<P, LOGC, KMAX, TW_SMEM, OTS>();
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
    PassArgs a;
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
        kern<<<dim3(tiles, cnt), T, smem, c.stream>>>(a);
    }
    return cudaGetLastError();
}

// Single pass over all n stages (n <= 12): one CTA per limb.
template <int N_LOG>
cudaError_t launch_single_n(const LaunchCtx& c, bool fwd)
{
    if (fwd)
        return launch_pass<N_LOG, 0, KMAX_ALL, true, true, 1, true, true, 0, false>(c, 0, nullptr, nullptr);
    return launch_pass<N_LOG, 0, KMAX_ALL, true, false, 1, true, true, 0, false>(c, 0, nullptr, nullptr);
}

// Two passes: P1 column-like stages [0, P1), then P2 row-like stages.
template <int P1, int P2, int LOGC_R, int KMAX_R, int OTS>
cudaError_t launch_two_pass_ots(const LaunchCtx& c, bool fwd)
{
    constexpr int LOGC_C = 4;
    constexpr int KMAX_C = KMAX_R;
    cudaError_t e;
    if (fwd) {
        e = launch_pass<P1, LOGC_C, KMAX_C, false, true, 1, false, true, 0, true>(c, 0, nullptr, nullptr);
        if (e != cudaSuccess) return e;
        constexpr int X2 = ct_range_after(1, P1);
        return launch_pass<P2, LOGC_R, KMAX_R, true, true, X2, true, false, OTS, false>(c, P1, c.ota_f, c.otb_f);
    }
    e = launch_pass<P2, LOGC_R, KMAX_R, true, false, 1, false, false, OTS, false>(c, P1, c.ota_i, c.otb_i);
    if (e != cudaSuccess) return e;
    constexpr int X1 = gs_range_after(1, P2);
    return launch_pass<P1, LOGC_C, KMAX_C, false, false, X1, true, true, 0, true>(c, 0, nullptr, nullptr);
}

// host helpers for the fused launch (fused_host.cu)
u32 fused_window_limbs(size_t limb_bytes);
cudaError_t encode_tile_maps(const LaunchCtx& c, int p1, int row_tile_words, CUtensorMap* mapC, CUtensorMap* mapR);
int device_sm_count();

template <int P1, int P2, int LOGC_R, int KMAX, bool FWD, int OTS>
cudaError_t launch_fused_dir(const LaunchCtx& c)
{
    using F = FusedCfg<P1, P2, LOGC_R, KMAX>;
    auto kern = ntt_fused_kernel<P1, P2, LOGC_R, KMAX, FWD, OTS>;
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
    if (!c.work || c.work_limbs < c.limbs) return cudaErrorInvalidValue;
    CUtensorMap mapC, mapR;
    cudaError_t e = encode_tile_maps(c, P1, F::TILE_R, &mapC, &mapR);
    if (e != cudaSuccess) return e;
    constexpr u32 UC = F::R2 / 16, UR = F::R1 / F::CR;
    const u64 units = (u64)c.limbs * (UC + UR);
    const u64 slots = (u64)device_sm_count() * (u64)occ;
    const u32 grid = (u32)(units < slots ? units : slots);
    FusedArgs a;
    a.primes = c.primes;
    a.tw = c.tw;
    a.ota = FWD ? c.ota_f : c.ota_i;
    a.otb = FWD ? c.otb_f : c.otb_i;
    a.ctl = c.work;
    a.status = c.status;
    a.tw_len = c.tw_len;
    a.L = c.L;
    a.limbs = c.limbs;
    a.a_window = fused_window_limbs(sizeof(u64) << (P1 + P2));
    a.max_polls = 1u << 22;
    kern<<<grid, F::THREADS, F::SMEM, c.stream>>>(mapC, mapR, a);
    return cudaGetLastError();
}

template <int P1, int P2, int LOGC_R, int KMAX, int OTS>
cudaError_t launch_fused(const LaunchCtx& c, bool fwd)
{
    return fwd ? launch_fused_dir<P1, P2, LOGC_R, KMAX, true, OTS>(c)
               : launch_fused_dir<P1, P2, LOGC_R, KMAX, false, OTS>(c);
}

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
    switch (c.ots) {
    case 0: return launch_fused<P1, P2, LOGC_R, KMAX_R, 0>(c, fwd);
    case 1: return launch_fused<P1, P2, LOGC_R, KMAX_R, 1>(c, fwd);
    case 2: return launch_fused<P1, P2, LOGC_R, KMAX_R, 2>(c, fwd);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ntt

// Internal plan object and kernel dispatch interface.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <vector>

#include "../../include/ntt_gb300.h"
#include "device_types.cuh"

namespace ntt {

// Pass split for N = 2^n: one pass for n <= SINGLE_PASS_MAX, else two passes
// of p1 = n - ceil(n/2) and p2 = ceil(n/2) stages.
constexpr int SINGLE_PASS_MAX = 12;
inline int split_p1(int n) { return n <= SINGLE_PASS_MAX ? n : n - (n + 1) / 2; }

// Everything a launch needs (device pointers are the plan's).
struct LaunchCtx {
    u64* data;
    u32 limbs;               // polynomials x primes covered by the launch
    u32 L;                   // primes per polynomial (limb l uses prime l % L)
    const PrimeDev* primes;
    const Tw* tw;
    u32 tw_len;
    const Tw* ota_f;
    const Tw* otb_f;
    const Tw* ota_i;
    const Tw* otb_i;
    u32 n;
    u32 p1;
    u32 ots;                 // OT stages (0 = table mode)
    cudaStream_t stream;
};

cudaError_t launch_transform(const LaunchCtx& c, bool fwd);
cudaError_t launch_pointwise(const PrimeDev* primes, u32 L, u32 n, const u64* a, const u64* b,
                             u64* out, u32 limbs, cudaStream_t s);

// per-n launchers (one translation unit each, compiled in parallel)
cudaError_t launch_single(const LaunchCtx& c, bool fwd);
cudaError_t launch_n13(const LaunchCtx& c, bool fwd);
cudaError_t launch_n14(const LaunchCtx& c, bool fwd);
cudaError_t launch_n15(const LaunchCtx& c, bool fwd);
cudaError_t launch_n16(const LaunchCtx& c, bool fwd);
cudaError_t launch_n17(const LaunchCtx& c, bool fwd);

}  // namespace ntt

struct ntt_plan {
    uint32_t N = 0, n = 0, L = 0;
    uint32_t p1 = 0, passes = 0;
    uint32_t twiddle_mode = 0, ot_stages = 0;
    int device = 0;
    std::vector<uint64_t> primes, psis;
    ntt::PrimeDev* d_primes = nullptr;
    ntt::Tw* d_tw = nullptr;
    uint32_t tw_len = 0;
    ntt::Tw* d_ota_f = nullptr;
    ntt::Tw* d_otb_f = nullptr;
    ntt::Tw* d_ota_i = nullptr;
    ntt::Tw* d_otb_i = nullptr;
    uint64_t device_bytes = 0;
    // staging for ntt_execute_host
    std::mutex stage_mu;
    uint64_t* d_stage = nullptr;
    size_t stage_bytes = 0;

    ntt::LaunchCtx ctx(uint64_t* data, uint32_t limbs, uint32_t Lused, cudaStream_t s) const
    {
        ntt::LaunchCtx c;
        c.data = reinterpret_cast<ntt::u64*>(data);
        c.limbs = limbs;
        c.L = Lused;
        c.primes = d_primes;
        c.tw = d_tw;
        c.tw_len = tw_len;
        c.ota_f = d_ota_f;
        c.otb_f = d_otb_f;
        c.ota_i = d_ota_i;
        c.otb_i = d_otb_i;
        c.n = n;
        c.p1 = p1;
        c.ots = twiddle_mode == NTT_TWIDDLE_OT ? ot_stages : 0;
        c.stream = s;
        return c;
    }
};

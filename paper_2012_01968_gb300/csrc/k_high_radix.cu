// The register-based high-radix organisation of Sec. VI-B: one kernel launch
// per group of k stages (radix 2^k per launch, the paper finds radix 16 best),
// each thread loading 2^k operands from global memory, running the k stages in
// registers and writing the results back.  Kept as a plan option
// (NTT_KERNEL_HIGH_RADIX) for the comparison of kernel organisations; like
// the radix-2 organisation it reads the table Psi in natural order.
//
// Launch for stages [s0, s0 + k): an item is 2^k elements spaced t = 2^{n-s0-k}
// apart, idx_i = b 2^{n-s0} + i t + j (block b < 2^{s0}, offset j < t).  At
// stage s0 + r, registers i and i + 2^{k-1-r} pair up, and the twiddle index
// idx >> (n - s) = (b << r) + (i >> (k - r)) is shared by each group of
// 2^{k-r} registers.
#include "arith.cuh"
#include "plan.h"

namespace ntt {

namespace {

template <int K, int r, int X>
__device__ __forceinline__ void hr_fwd(u64 (&x)[1 << K], const Tw* __restrict__ tw, const u32 s0, const u32 b,
                                       const u64 q, const u64 q4)
{
    if constexpr (r < K) {
        constexpr int h = 1 << (K - 1 - r);
        const u32 s = s0 + (u32)r;
#pragma unroll
        for (int g = 0; g < (1 << r); ++g) {
            const Tw w = tw[(1u << s) + (b << r) + (u32)g];
#pragma unroll
            for (int i = 0; i < h; ++i) ct_bfly<X>(x[g * 2 * h + i], x[g * 2 * h + i + h], w.w, w.wp, q, q4);
        }
        hr_fwd<K, r + 1, ct_next(X)>(x, tw, s0, b, q, q4);
    }
}

// Gentleman-Sande stages r = K-1 .. 0; S0: the group holds global stage 0,
// whose butterfly also applies N^{-1} (b == 0 there).
template <int K, int r, int X, bool S0>
__device__ __forceinline__ void hr_inv(u64 (&x)[1 << K], const Tw* __restrict__ tw, const u32 s0, const u32 b,
                                       const PrimeDev& pr, const u64 q)
{
    if constexpr (r >= 0) {
        constexpr int h = 1 << (K - 1 - r);
        static_assert(X <= 8, "GS inputs must stay below 8q");
        if constexpr (S0 && r == 0) {
#pragma unroll
            for (int i = 0; i < h; ++i) gs_bfly_scaled<X, true>(x[i], x[i + h], pr.w1ninv, pr.ninv, q);
        } else {
            const u32 s = s0 + (u32)r;
#pragma unroll
            for (int g = 0; g < (1 << r); ++g) {
                // Psi^{-1}[2^s + jj] = -Psi[2^{s+1} - 1 - jj]
                const u32 jj = (b << r) + (u32)g;
                const Tw w = tw[(2u << s) - 1u - jj];
#pragma unroll
                for (int i = 0; i < h; ++i) gs_bfly<X, true>(x[g * 2 * h + i], x[g * 2 * h + i + h], w.w, w.wp, q);
            }
        }
        hr_inv<K, r - 1, gs_next(X), S0>(x, tw, s0, b, pr, q);
    }
}

template <bool FWD, int K, bool S0>
__global__ void __launch_bounds__(256) high_radix_kernel(u64* __restrict__ data, const PrimeDev* __restrict__ primes,
                                                       const Tw* __restrict__ tw, u32 tw_len, u32 L, u32 n, u32 s0,
                                                       u64 total)
{
    constexpr int E = 1 << K;
    const u32 nb = n - s0 - (u32)K;                  // log2 of the spacing t
    const u32 per_limb = 1u << (n - (u32)K);         // items per limb
    for (u64 m = blockIdx.x * (u64)blockDim.x + threadIdx.x; m < total; m += (u64)gridDim.x * blockDim.x) {
        const u64 limb = m >> (n - (u32)K);
        const u32 mi = (u32)m & (per_limb - 1u);
        const u32 b = mi >> nb, j = mi & ((1u << nb) - 1u);
        const u32 base = (b << (n - s0)) + j;
        const u32 pi = (u32)(limb % L);
        const PrimeDev& pr = primes[pi];
        const u64 q = pr.q;
        const Tw* t = tw + (size_t)pi * tw_len;
        u64* d = data + (limb << n);
        u64 x[E];
        if (nb == 0 && E >= 2) {
            // the item is 2^K consecutive words (16-byte aligned: base is a multiple of 2^K)
#pragma unroll
            for (int i = 0; i < E; i += 2) {
                const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(d + base + i);
                x[i] = v.x;
                x[i + 1] = v.y;
            }
        } else {
#pragma unroll
            for (int i = 0; i < E; ++i) x[i] = d[base + ((u32)i << nb)];
        }
        if constexpr (FWD) {
            hr_fwd<K, 0, 1>(x, t, s0, b, q, q << 2);
#pragma unroll
            for (int i = 0; i < E; ++i) x[i] = canon<ct_range_after(1, K)>(x[i], q, pr.rc, pr.rsh);
        } else {
            hr_inv<K, K - 1, 1, S0>(x, t, s0, b, pr, q);
            constexpr int XO = S0 ? 4 : gs_range_after(1, K);
#pragma unroll
            for (int i = 0; i < E; ++i) x[i] = canon<XO>(x[i], q, pr.rc, pr.rsh);
        }
        if (nb == 0 && E >= 2) {
#pragma unroll
            for (int i = 0; i < E; i += 2)
                *reinterpret_cast<ulonglong2*>(d + base + i) = make_ulonglong2(x[i], x[i + 1]);
        } else {
#pragma unroll
            for (int i = 0; i < E; ++i) d[base + ((u32)i << nb)] = x[i];
        }
    }
}

template <bool FWD, int K>
cudaError_t launch_group(const LaunchCtx& c, u32 s0, u32 blocks, u64 total)
{
    if (!FWD && s0 == 0)
        high_radix_kernel<FWD, K, true><<<blocks, 256, 0, c.stream>>>(c.data, c.primes, c.tw, c.tw_len, c.L, c.n, s0,
                                                                      total);
    else
        high_radix_kernel<FWD, K, false><<<blocks, 256, 0, c.stream>>>(c.data, c.primes, c.tw, c.tw_len, c.L, c.n,
                                                                       s0, total);
    return cudaGetLastError();
}

template <bool FWD>
cudaError_t launch_group_k(const LaunchCtx& c, u32 s0, u32 k)
{
    const u64 total = (u64)c.limbs << (c.n - k);
    u64 blocks = (total + 255) / 256;
    const u64 cap = 152ull * 16;
    if (blocks > cap) blocks = cap;
    switch (k) {
    case 1: return launch_group<FWD, 1>(c, s0, (u32)blocks, total);
    case 2: return launch_group<FWD, 2>(c, s0, (u32)blocks, total);
    case 3: return launch_group<FWD, 3>(c, s0, (u32)blocks, total);
    case 4: return launch_group<FWD, 4>(c, s0, (u32)blocks, total);
    case 5: return launch_group<FWD, 5>(c, s0, (u32)blocks, total);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_high_radix(const LaunchCtx& c, bool fwd)
{
    if (c.limbs == 0) return cudaSuccess;
    const u32 k = c.high_radix, n = c.n;
    if (k < 1 || k > 5) return cudaErrorInvalidValue;
    const u32 groups = (n + k - 1) / k;
    for (u32 r = 0; r < groups; ++r) {
        const u32 g = fwd ? r : groups - 1 - r;           // the inverse runs the groups in reverse
        const u32 s0 = g * k, kk = n - s0 < k ? n - s0 : k;
        const cudaError_t e = fwd ? launch_group_k<true>(c, s0, kk) : launch_group_k<false>(c, s0, kk);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace ntt

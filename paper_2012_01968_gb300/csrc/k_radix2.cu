// The radix-2 organisation the paper starts from (Sec. VI): one kernel
// launch per stage, one thread per butterfly, operands and twiddles in global
// memory, canonical residues between stages.  Kept as a plan option
// (NTT_KERNEL_RADIX2) for comparison with the tiled kernels; it reads the
// table Psi in natural order (Psi[2^s + j] at index 2^s + j).
#include "arith.cuh"
#include "plan.h"

namespace ntt {

namespace {

__device__ __forceinline__ u64 canon4(u64 x, u64 q) { return csub(csub(x, q << 1), q); }   // [0, 4q) -> [0, q)

// Stage s: 2^s groups of span t = 2^{n-1-s}; butterfly b = j t + k pairs
// elements j 2t + k and j 2t + k + t.
template <bool FWD>
__global__ void __launch_bounds__(256) radix2_stage_kernel(u64* __restrict__ data, const PrimeDev* __restrict__ primes,
                                                         const Tw* __restrict__ tw, u32 tw_len, u32 L, u32 n, u32 s,
                                                         u64 total, bool scale)
{
    const u32 half = 1u << (n - 1), t = half >> s;
    for (u64 idx = blockIdx.x * (u64)blockDim.x + threadIdx.x; idx < total; idx += (u64)gridDim.x * blockDim.x) {
        const u64 limb = idx >> (n - 1);
        const u32 b = (u32)(idx & (half - 1));
        const u32 j = b >> (n - 1 - s), k = b & (t - 1);
        const u32 i0 = (j << (n - s)) + k, i1 = i0 + t;
        const u32 pi = (u32)(limb % L);
        const PrimeDev& pr = primes[pi];
        const u64 q = pr.q;
        u64* d = data + (limb << n);
        const u64 x = d[i0], y = d[i1];
        if (FWD) {
            const Tw w = tw[(size_t)pi * tw_len + (1u << s) + j];
            const u64 v = canon4(shoup_lazy(y, w.w, w.wp, q), q);
            d[i0] = csub(x + v, q);
            d[i1] = csub(x + q - v, q);
        } else {
            // Psi^{-1}[2^s + j] = -Psi[2^{s+1} - 1 - j]: the difference is taken as y - x
            const u64 sum = csub(x + y, q), dif = csub(y + q - x, q);
            if (scale) {                      // s = 0: N^{-1} folded into both outputs
                d[i0] = canon4(shoup_lazy(sum, pr.ninv.w, pr.ninv.wp, q), q);
                d[i1] = canon4(shoup_lazy(dif, pr.w1ninv.w, pr.w1ninv.wp, q), q);
            } else {
                const Tw w = tw[(size_t)pi * tw_len + (2u << s) - 1u - j];
                d[i0] = sum;
                d[i1] = canon4(shoup_lazy(dif, w.w, w.wp, q), q);
            }
        }
    }
}

}  // namespace

cudaError_t launch_radix2(const LaunchCtx& c, bool fwd)
{
    const u64 total = (u64)c.limbs << (c.n - 1);
    if (total == 0) return cudaSuccess;
    constexpr u32 T = 256;
    u64 blocks = (total + T - 1) / T;
    const u64 cap = 152ull * 64;
    if (blocks > cap) blocks = cap;
    for (u32 r = 0; r < c.n; ++r) {
        const u32 s = fwd ? r : c.n - 1 - r;
        if (fwd)
            radix2_stage_kernel<true><<<(u32)blocks, T, 0, c.stream>>>(c.data, c.primes, c.tw, c.tw_len, c.L, c.n, s,
                                                                        total, false);
        else
            radix2_stage_kernel<false><<<(u32)blocks, T, 0, c.stream>>>(c.data, c.primes, c.tw, c.tw_len, c.L, c.n, s,
                                                                         total, s == 0);
    }
    return cudaGetLastError();
}

}  // namespace ntt

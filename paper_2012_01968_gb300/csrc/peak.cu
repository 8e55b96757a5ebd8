// Butterfly rate of the integer multiply pipe, for the roofline of the
// transform kernels (not part of the transform path): a register-only loop of
// the forward butterfly with Shoup's lazy product, 16 values per thread in
// four radix-2 stages per round, the reduction of the value range every
// other stage as in the transform kernels.  The values are not meaningful.
#include <cuda_runtime.h>

#include "arith.cuh"
#include "ntt_gb300.h"

extern "C" void ntt_internal_set_cuda_error(cudaError_t e);

namespace {

using namespace ntt;

__global__ void __launch_bounds__(256) bfly_rate_kernel(u64* out, u64 q, u64 w0, u64 wp0, u32 rounds)
{
    const u64 q4 = q << 2;
    u64 x[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) x[i] = (u64)(threadIdx.x * 16u + i + 1u);
    for (u32 r = 0; r < rounds; ++r) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int half = 16 >> (k + 1);
#pragma unroll
            for (int pre = 0; pre < (1 << k); ++pre) {
                const u64 w = w0 + (u64)(pre + k) + r, wp = wp0 ^ (u64)pre;   // vary, so nothing is hoisted
#pragma unroll
                for (int i = 0; i < half; ++i) {
                    const int a = pre * 2 * half + i;
                    if (k & 1) ct_bfly<16>(x[a], x[a + half], w, wp, q, q4);
                    else ct_bfly<12>(x[a], x[a + half], w, wp, q, q4);
                }
            }
        }
    }
    u64 s = 0;
#pragma unroll
    for (int i = 0; i < 16; ++i) s ^= x[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" ntt_status ntt_measure_butterfly_rate(double* gbfly_per_s)
{
    if (!gbfly_per_s) return NTT_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned grid = (unsigned)(sms > 0 ? sms : 1) * 8u, threads = 256u, rounds = 512u;
    u64* out = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(u64) * grid * threads);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    const u64 q = 1152921504606584833ull;                 // 2^60 - 2^18 + 1
    const u64 w = 123456789123ull, wp = (u64)(((unsigned __int128)w << 64) / q);
    float ms = 0;
    if (e == cudaSuccess) {
        bfly_rate_kernel<<<grid, threads>>>(out, q, w, wp, rounds);      // warm-up
        cudaEventRecord(a);
        for (int i = 0; i < 5; ++i) bfly_rate_kernel<<<grid, threads>>>(out, q, w, wp, rounds);
        cudaEventRecord(b);
        e = cudaEventSynchronize(b);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaFree(out);
    if (e != cudaSuccess || ms <= 0) {
        ntt_internal_set_cuda_error(e);
        cudaGetLastError();
        return NTT_ERR_CUDA;
    }
    const double bfly = 5.0 * grid * threads * rounds * 32.0;             // 4 stages x 8 per round
    *gbfly_per_s = bfly / (ms * 1e-3) / 1e9;
    return NTT_OK;
}

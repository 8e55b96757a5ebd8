// C ABI entry points (include/ntt_gb300.h) and the pointwise product kernel.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>

#include "arith.cuh"
#include "plan.h"

namespace {
thread_local char g_cuda_err[256] = "no error";
}

cudaError_t ntt_internal_grow_work(ntt_plan* p, uint32_t limbs);

extern "C" void ntt_internal_set_cuda_error(cudaError_t e)
{
    std::snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
}

namespace ntt {

cudaError_t launch_transform(const LaunchCtx& c, bool fwd)
{
    if (c.limbs == 0) return cudaSuccess;
    if (c.n <= (u32)SINGLE_PASS_MAX) return launch_single(c, fwd);
    switch (c.n) {
    case 13: return launch_n13(c, fwd);
    case 14: return launch_n14(c, fwd);
    case 15: return launch_n15(c, fwd);
    case 16: return launch_n16(c, fwd);
    case 17: return launch_n17(c, fwd);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fused_jobs(const JobsCtx& c, bool fwd)
{
    switch (c.n) {
    case 13: return launch_jobs_n13(c, fwd);
    case 14: return launch_jobs_n14(c, fwd);
    case 15: return launch_jobs_n15(c, fwd);
    case 16: return launch_jobs_n16(c, fwd);
    case 17: return launch_jobs_n17(c, fwd);
    default: return cudaErrorInvalidValue;
    }
}

// c = a * b mod q_l, two words per thread per step, canonical output.
__global__ void __launch_bounds__(256) pointwise_kernel(const PrimeDev* __restrict__ primes, u32 L, u32 n,
                                                        const u64* __restrict__ a, const u64* __restrict__ b,
                                                        u64* __restrict__ out, u32 limbs)
{
    const u32 half_n = (1u << n) >> 1;         // vectors per limb
    const size_t total = (size_t)limbs * half_n;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const u32 limb = (u32)(i >> (n - 1));
        const PrimeDev& p = primes[limb % L];
        const ulonglong2 x = reinterpret_cast<const ulonglong2*>(a)[i];
        const ulonglong2 y = reinterpret_cast<const ulonglong2*>(b)[i];
        ulonglong2 r;
        r.x = canon<3>(mulmod_barrett(x.x, y.x, p.q, p.mu, p.k), p.q, p.mbar);
        r.y = canon<3>(mulmod_barrett(x.y, y.y, p.q, p.mu, p.k), p.q, p.mbar);
        reinterpret_cast<ulonglong2*>(out)[i] = r;
    }
}

cudaError_t launch_pointwise(const PrimeDev* primes, u32 L, u32 n, const u64* a, const u64* b, u64* out,
                             u32 limbs, cudaStream_t s)
{
    const size_t total = ((size_t)limbs << n) / 2;
    if (total == 0) return cudaSuccess;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    size_t blocks = (total + 255) / 256;
    const size_t cap = (size_t)sms * 8;
    if (blocks > cap) blocks = cap;
    pointwise_kernel<<<(unsigned)blocks, 256, 0, s>>>(primes, L, n, a, b, out, limbs);
    return cudaGetLastError();
}

}  // namespace ntt

namespace {

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

ntt_status to_status(cudaError_t e)
{
    if (e == cudaSuccess) return NTT_OK;
    ntt_internal_set_cuda_error(e);
    return e == cudaErrorMemoryAllocation ? NTT_ERR_OOM : NTT_ERR_CUDA;
}

ntt_status transform(const ntt_plan* p, uint64_t* data, uint32_t batch, uint32_t levels, void* stream,
                     bool fwd)
{
    if (!p || !data || batch == 0 || levels == 0 || levels > p->L) return NTT_ERR_INVALID_ARG;
    if (!aligned16(data)) return NTT_ERR_MISALIGNED;
    const uint64_t limbs = (uint64_t)batch * levels;
    if (limbs > 0xFFFFFFFFull) return NTT_ERR_INVALID_ARG;
    if (p->passes == 2 && p->kernel == NTT_KERNEL_FUSED && p->work_limbs < limbs) {
        cudaError_t e = ntt_internal_grow_work(const_cast<ntt_plan*>(p), (uint32_t)limbs);
        if (e != cudaSuccess) return to_status(e);
    }
    const ntt::LaunchCtx c = p->ctx(data, (uint32_t)limbs, levels, (cudaStream_t)stream);
    return to_status(ntt::launch_transform(c, fwd));
}

}  // namespace

extern "C" {

ntt_status ntt_forward(const ntt_plan* p, uint64_t* data, uint32_t batch, void* stream)
{
    return transform(p, data, batch, p ? p->L : 0, stream, true);
}

ntt_status ntt_inverse(const ntt_plan* p, uint64_t* data, uint32_t batch, void* stream)
{
    return transform(p, data, batch, p ? p->L : 0, stream, false);
}

ntt_status ntt_forward_levels(const ntt_plan* p, uint64_t* data, uint32_t batch, uint32_t levels,
                              void* stream)
{
    return transform(p, data, batch, levels, stream, true);
}

ntt_status ntt_inverse_levels(const ntt_plan* p, uint64_t* data, uint32_t batch, uint32_t levels,
                              void* stream)
{
    return transform(p, data, batch, levels, stream, false);
}

ntt_status ntt_mul_pointwise(const ntt_plan* p, const uint64_t* a, const uint64_t* b, uint64_t* c,
                             uint32_t batch, void* stream)
{
    if (!p || !a || !b || !c || batch == 0) return NTT_ERR_INVALID_ARG;
    if (!aligned16(a) || !aligned16(b) || !aligned16(c)) return NTT_ERR_MISALIGNED;
    const uint64_t limbs = (uint64_t)batch * p->L;
    if (limbs > 0xFFFFFFFFull) return NTT_ERR_INVALID_ARG;
    return to_status(ntt::launch_pointwise(p->d_primes, p->L, p->n, reinterpret_cast<const ntt::u64*>(a),
                                           reinterpret_cast<const ntt::u64*>(b), reinterpret_cast<ntt::u64*>(c),
                                           (uint32_t)limbs,
                                           (cudaStream_t)stream));
}

ntt_status ntt_execute_host(const ntt_plan* cp, const uint64_t* host_in, uint64_t* host_out, uint32_t batch,
                            uint32_t ops, void* stream)
{
    if (!cp || !host_in || !host_out || batch == 0) return NTT_ERR_INVALID_ARG;
    if (ops == 0 || (ops & ~(uint32_t)(NTT_OP_FORWARD | NTT_OP_INVERSE))) return NTT_ERR_INVALID_ARG;
    ntt_plan* p = const_cast<ntt_plan*>(cp);
    const size_t bytes = (size_t)batch * p->L * p->N * sizeof(uint64_t);
    std::lock_guard<std::mutex> g(p->stage_mu);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (p->stage_bytes < bytes) {
        if (p->d_stage) {
            e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return to_status(e);
            cudaFree(p->d_stage);
            p->d_stage = nullptr;
            p->stage_bytes = 0;
        }
        e = cudaMalloc(&p->d_stage, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return to_status(e);
        }
        p->stage_bytes = bytes;
    }
    e = cudaMemcpyAsync(p->d_stage, host_in, bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return to_status(e);
    if (p->passes == 2 && p->kernel == NTT_KERNEL_FUSED && p->work_limbs < batch * p->L) {
        e = ntt_internal_grow_work(p, batch * p->L);
        if (e != cudaSuccess) return to_status(e);
    }
    const ntt::LaunchCtx c = p->ctx(p->d_stage, batch * p->L, p->L, s);
    if (ops & NTT_OP_FORWARD) {
        e = ntt::launch_transform(c, true);
        if (e != cudaSuccess) return to_status(e);
    }
    if (ops & NTT_OP_INVERSE) {
        e = ntt::launch_transform(c, false);
        if (e != cudaSuccess) return to_status(e);
    }
    e = cudaMemcpyAsync(host_out, p->d_stage, bytes, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return to_status(e);
    return to_status(cudaStreamSynchronize(s));
}

const char* ntt_status_string(ntt_status s)
{
    switch (s) {
    case NTT_OK: return "NTT_OK";
    case NTT_ERR_INVALID_ARG: return "NTT_ERR_INVALID_ARG: invalid argument";
    case NTT_ERR_BAD_PRIME: return "NTT_ERR_BAD_PRIME: modulus is not a prime = 1 mod 2N in (2^32, 2^60)";
    case NTT_ERR_MISALIGNED: return "NTT_ERR_MISALIGNED: device pointer not 16-byte aligned";
    case NTT_ERR_CUDA: return "NTT_ERR_CUDA: CUDA runtime error";
    case NTT_ERR_OOM: return "NTT_ERR_OOM: out of memory";
    case NTT_ERR_BUSY: return "NTT_ERR_BUSY: admission refused";
    case NTT_ERR_TIMEOUT: return "NTT_ERR_TIMEOUT: bounded wait expired";
    case NTT_ERR_DEVICE: return "NTT_ERR_DEVICE: kernel reported an error";
    case NTT_ERR_LIMIT: return "NTT_ERR_LIMIT: batch * levels exceeds the fixed work area of the no-allocation call";
    }
    return "unknown ntt_status";
}

const char* ntt_last_cuda_error(void) { return g_cuda_err; }

}  // extern "C"

// C ABI entry points (include/ntt_gb300.h) and the pointwise product kernel.
#include <cuda_runtime.h>

#include <cstdio>
#include <vector>
#include <cstring>

#include "arith.cuh"
#include "host_logic.h"
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
    if (c.cluster) return launch_cluster(c, fwd);
    if (c.radix2) return launch_radix2(c, fwd);
    if (c.high_radix) return launch_high_radix(c, fwd);
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
        r.x = canon<3>(mulmod_barrett(x.x, y.x, p.q, p.mu, p.k), p.q, p.rc, p.rsh);
        r.y = canon<3>(mulmod_barrett(x.y, y.y, p.q, p.mu, p.k), p.q, p.rc, p.rsh);
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

// Whether forward + inverse of a plan runs as one launch (fused two-pass
// plans and cluster plans).
bool chains(const ntt_plan* p)
{
    return (p->passes == 2 && p->kernel == NTT_KERNEL_FUSED) || p->kernel == NTT_KERNEL_CLUSTER;
}

// The operations `ops` (NTT_OP_*) on one launch context: forward + inverse as
// one chained launch where the plan allows it, else one call per direction.
cudaError_t launch_ops(const ntt_plan* p, ntt::LaunchCtx c, uint32_t ops)
{
    if (ops == (NTT_OP_FORWARD | NTT_OP_INVERSE) && chains(p)) {
        c.chain = 1;
        return ntt::launch_transform(c, true);
    }
    cudaError_t e = cudaSuccess;
    if (ops & NTT_OP_FORWARD) e = ntt::launch_transform(c, true);
    if (e == cudaSuccess && (ops & NTT_OP_INVERSE)) e = ntt::launch_transform(c, false);
    return e;
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

ntt_status ntt_execute(const ntt_plan* p, uint64_t* data, uint32_t batch, uint32_t ops, void* stream)
{
    if (!p || !data || batch == 0) return NTT_ERR_INVALID_ARG;
    if (ops == 0 || (ops & ~(uint32_t)(NTT_OP_FORWARD | NTT_OP_INVERSE))) return NTT_ERR_INVALID_ARG;
    if (!aligned16(data)) return NTT_ERR_MISALIGNED;
    const uint64_t limbs = (uint64_t)batch * p->L;
    if (limbs > 0xFFFFFFFFull) return NTT_ERR_INVALID_ARG;
    const bool chain = ops == (NTT_OP_FORWARD | NTT_OP_INVERSE) && chains(p);
    const uint64_t need = chain ? ntt::chain_work_limbs(limbs) : limbs;
    if (need > 0xFFFFFFFFull) return NTT_ERR_INVALID_ARG;
    if (p->passes == 2 && p->kernel == NTT_KERNEL_FUSED && p->work_limbs < need) {
        cudaError_t e = ntt_internal_grow_work(const_cast<ntt_plan*>(p), (uint32_t)need);
        if (e != cudaSuccess) return to_status(e);
    }
    const ntt::LaunchCtx c = p->ctx(data, (uint32_t)limbs, p->L, (cudaStream_t)stream);
    return to_status(launch_ops(p, c, ops));
}

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

ntt_status ntt_mul_negacyclic(const ntt_plan* p, uint64_t* a, uint64_t* b, uint64_t* c, uint32_t batch,
                              void* stream)
{
    if (!p || !a || !b || !c || batch == 0 || a == b) return NTT_ERR_INVALID_ARG;
    if (!aligned16(a) || !aligned16(b) || !aligned16(c)) return NTT_ERR_MISALIGNED;
    const uint64_t limbs = (uint64_t)batch * p->L;
    if (2 * limbs > 0x7FFFFFFFull) return NTT_ERR_INVALID_ARG;
    const size_t bytes = (size_t)limbs * p->N * sizeof(uint64_t);
    const uintptr_t pa = (uintptr_t)a, pb = (uintptr_t)b;
    if (pa < pb + bytes && pb < pa + bytes) return NTT_ERR_INVALID_ARG;    // a and b overlap
    const cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (p->passes == 2 && p->kernel == NTT_KERNEL_FUSED) {
        // both forward transforms in one launch of the fused kernel (two jobs)
        if (p->work_limbs < 2 * limbs) {
            e = ntt_internal_grow_work(const_cast<ntt_plan*>(p), (uint32_t)(2 * limbs));
            if (e != cudaSuccess) return to_status(e);
        }
        const ntt::JobCtx ja{reinterpret_cast<ntt::u64*>(a), (uint32_t)limbs, p->L, p->d_primes, p->d_tw, p->tw_len,
                             p->d_ota_f, p->d_otb_f, p->d_ota_i, p->d_otb_i};
        ntt::JobCtx jb = ja;
        jb.data = reinterpret_cast<ntt::u64*>(b);
        const ntt::JobCtx jobs[2] = {ja, jb};
        const uint32_t ots = p->twiddle_mode == NTT_TWIDDLE_OT ? p->ot_stages : 0;
        const ntt::JobsCtx jc{jobs, 2u, p->n, ots, p->d_status, p->d_work, p->work_limbs, s, 0u, p->geom};
        e = ntt::launch_fused_jobs(jc, true);
        if (e != cudaSuccess) return to_status(e);
        if (c == a || c == b) {
            // the product in place: the inverse's first pass multiplies each
            // tile of c by the other factor before its stages (no separate
            // element-wise pass over the data)
            ntt::LaunchCtx ci = p->ctx(c, (uint32_t)limbs, p->L, s);
            ci.mulb = reinterpret_cast<const ntt::u64*>(c == a ? b : a);
            return to_status(ntt::launch_transform(ci, false));
        }
    } else {
        const ntt::LaunchCtx ca = p->ctx(a, (uint32_t)limbs, p->L, s);
        e = ntt::launch_transform(ca, true);
        if (e == cudaSuccess) e = ntt::launch_transform(p->ctx(b, (uint32_t)limbs, p->L, s), true);
    }
    if (e == cudaSuccess)
        e = ntt::launch_pointwise(p->d_primes, p->L, p->n, reinterpret_cast<const ntt::u64*>(a),
                                  reinterpret_cast<const ntt::u64*>(b), reinterpret_cast<ntt::u64*>(c),
                                  (uint32_t)limbs, s);
    if (e == cudaSuccess) e = ntt::launch_transform(p->ctx(c, (uint32_t)limbs, p->L, s), false);
    return to_status(e);
}

// Enqueue the host-buffer pipeline of ntt_execute_host / _async; the
// caller's stream waits for the last copy-out.  `wait` drains the plan's host
// streams before returning (the synchronous call).
static ntt_status host_pipeline(const ntt_plan* cp, const uint64_t* host_in, uint64_t* host_out, uint32_t batch,
                                uint32_t ops, void* stream, bool wait)
{
    if (!cp || !host_in || !host_out || batch == 0) return NTT_ERR_INVALID_ARG;
    if (ops == 0 || (ops & ~(uint32_t)(NTT_OP_FORWARD | NTT_OP_INVERSE))) return NTT_ERR_INVALID_ARG;
    ntt_plan* p = const_cast<ntt_plan*>(cp);
    const uint64_t limbs64 = (uint64_t)batch * p->L;
    if (limbs64 > 0x7FFFFFFFull) return NTT_ERR_INVALID_ARG;
    const uint32_t L = p->L;
    const size_t N = p->N;
    const size_t bytes = (size_t)limbs64 * N * sizeof(uint64_t);

    // Segments of the data: a limb range inside one polynomial (tables viewed
    // from its first prime), or a group of whole polynomials.  All segments
    // are copied in back to back on one stream, transformed on the compute
    // streams as soon as their copy has landed, and copied out on another
    // stream as soon as their transforms are done, so the two copy directions
    // and the transforms overlap.
    // (an asynchronous call takes fewer, larger segments: its copies overlap
    // the neighbouring calls' work, and larger launches run more efficiently)
    using Seg = ntt::host::Segment;
    constexpr uint32_t kSegments = ntt_plan::kHostSegments;
    const std::vector<Seg> segs =
        ntt::host::split_segments(batch, L, wait ? kSegments : (uint32_t)ntt_plan::kHostSegmentsAsync);
    if (segs.size() > kSegments) return NTT_ERR_INVALID_ARG;      // cannot happen: one event pair per segment
    uint32_t seg_max = 0;
    for (const Seg& g : segs) seg_max = g.count > seg_max ? g.count : seg_max;

    std::lock_guard<std::mutex> g(p->stage_mu);
    cudaError_t e = cudaSuccess;
    auto mk_stream = [&](cudaStream_t& st) {
        if (e == cudaSuccess && !st) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    };
    auto mk_event = [&](cudaEvent_t& ev) {
        if (e == cudaSuccess && !ev) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    };
    mk_stream(p->h_in);
    mk_stream(p->h_out);
    for (int k = 0; k < ntt_plan::kHostCompute; ++k) mk_stream(p->h_comp[k]);
    mk_event(p->hfork);
    mk_event(p->h_join);
    for (uint32_t k = 0; k < kSegments; ++k) {
        mk_event(p->h_loaded[k]);
        mk_event(p->h_done[k]);
        for (int b = 0; b < ntt_plan::kHostBuffers; ++b) mk_event(p->h_out_done[b][k]);
    }
    if (e != cudaSuccess) return to_status(e);
    auto drain = [&]() {
        cudaError_t se = cudaStreamSynchronize(p->h_in);
        for (int k = 0; k < ntt_plan::kHostCompute; ++k) {
            const cudaError_t sk = cudaStreamSynchronize(p->h_comp[k]);
            if (se == cudaSuccess) se = sk;
        }
        const cudaError_t so = cudaStreamSynchronize(p->h_out);
        return se == cudaSuccess ? so : se;
    };
    // a chained forward + inverse launch needs the larger work area
    const uint32_t work_need = ops == (NTT_OP_FORWARD | NTT_OP_INVERSE) && chains(p)
                                   ? (uint32_t)ntt::chain_work_limbs(seg_max) : seg_max;
    if (p->stage_bytes < bytes || p->hwork_limbs < work_need) {
        // earlier asynchronous calls may still use the staging: drain first
        e = drain();
        if (e != cudaSuccess) return to_status(e);
        cudaFree(p->d_stage);
        cudaFree(p->d_hwork);
        p->d_stage = nullptr;
        p->d_hwork = nullptr;
        p->stage_bytes = 0;
        p->hwork_limbs = 0;
        for (int b = 0; b < ntt_plan::kHostBuffers; ++b) p->h_prev_segs[b] = 0;
        const size_t wwords = ntt::fused_work_words(work_need) * ntt_plan::kHostCompute;
        e = cudaMalloc(&p->d_stage, bytes * ntt_plan::kHostBuffers);
        if (e == cudaSuccess) e = cudaMalloc(&p->d_hwork, wwords * sizeof(uint32_t));
        if (e == cudaSuccess) e = cudaMemset(p->d_hwork, 0, wwords * sizeof(uint32_t));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return to_status(e);
        }
        p->stage_bytes = bytes;
        p->hwork_limbs = work_need;
    }

    // this call's staging buffer (alternate calls use alternate buffers)
    const uint32_t sb = p->h_next;
    p->h_next = (sb + 1) % ntt_plan::kHostBuffers;
    uint64_t* const stage = p->d_stage + (p->stage_bytes / sizeof(uint64_t)) * sb;

    // after the caller's earlier work on `stream`
    e = cudaEventRecord(p->hfork, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->h_in, p->hfork, 0);
    for (size_t i = 0; i < segs.size() && e == cudaSuccess; ++i) {
        const size_t off = (size_t)segs[i].first * N, nbytes = (size_t)segs[i].count * N * sizeof(uint64_t);
        // the staging range must have been copied out by the buffer's previous call
        for (uint32_t j = 0; j < p->h_prev_segs[sb] && e == cudaSuccess; ++j) {
            const uint32_t a0 = p->h_prev_first[sb][j], a1 = a0 + p->h_prev_count[sb][j];
            if (a0 < segs[i].first + segs[i].count && segs[i].first < a1)
                e = cudaStreamWaitEvent(p->h_in, p->h_out_done[sb][j], 0);
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(stage + off, host_in + off, nbytes, cudaMemcpyHostToDevice, p->h_in);
        if (e == cudaSuccess) e = cudaEventRecord(p->h_loaded[i], p->h_in);
    }
    for (size_t i = 0; i < segs.size() && e == cudaSuccess; ++i) {
        const Seg& sg = segs[i];
        const int k = (int)(i % ntt_plan::kHostCompute);
        cudaStream_t s = p->h_comp[k];
        const size_t off = (size_t)sg.first * N;
        e = cudaStreamWaitEvent(s, p->h_loaded[i], 0);
        if (e != cudaSuccess) break;
        ntt::LaunchCtx c = p->ctx_range(stage + off, sg.count, sg.lview, sg.prime0, s);
        c.work = p->d_hwork + ntt::fused_work_words(p->hwork_limbs) * (size_t)k;
        c.work_limbs = p->hwork_limbs;
        e = launch_ops(p, c, ops);
        if (e == cudaSuccess) e = cudaEventRecord(p->h_done[i], s);
    }
    for (size_t i = 0; i < segs.size() && e == cudaSuccess; ++i) {
        const size_t off = (size_t)segs[i].first * N, nbytes = (size_t)segs[i].count * N * sizeof(uint64_t);
        e = cudaStreamWaitEvent(p->h_out, p->h_done[i], 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(host_out + off, stage + off, nbytes, cudaMemcpyDeviceToHost, p->h_out);
        if (e == cudaSuccess) e = cudaEventRecord(p->h_out_done[sb][i], p->h_out);
    }
    if (e == cudaSuccess) {
        for (size_t i = 0; i < segs.size(); ++i) {
            p->h_prev_first[sb][i] = segs[i].first;
            p->h_prev_count[sb][i] = segs[i].count;
        }
        p->h_prev_segs[sb] = (uint32_t)segs.size();
        e = cudaEventRecord(p->h_join, p->h_out);
        if (e == cudaSuccess) e = cudaStreamWaitEvent((cudaStream_t)stream, p->h_join, 0);
    }
    if (!wait && e == cudaSuccess) return NTT_OK;
    // drain every stream, also after an error, before the staging can be reused
    const cudaError_t se = drain();
    if (e != cudaSuccess) p->h_prev_segs[sb] = 0;
    if (e != cudaSuccess || se != cudaSuccess) return to_status(e != cudaSuccess ? e : se);
    // a bounded wait of the kernels that ran out (left set for ntt_plan_device_status)
    uint32_t dev_status = 0;
    e = cudaMemcpy(&dev_status, p->d_status, sizeof(dev_status), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return to_status(e);
    return dev_status ? NTT_ERR_DEVICE : NTT_OK;
}

ntt_status ntt_execute_host(const ntt_plan* cp, const uint64_t* host_in, uint64_t* host_out, uint32_t batch,
                            uint32_t ops, void* stream)
{
    return host_pipeline(cp, host_in, host_out, batch, ops, stream, true);
}

ntt_status ntt_execute_host_async(const ntt_plan* cp, const uint64_t* host_in, uint64_t* host_out, uint32_t batch,
                                  uint32_t ops, void* stream)
{
    return host_pipeline(cp, host_in, host_out, batch, ops, stream, false);
}

// Test hook (not part of the public interface): the forward transform with
// the first-pass queue of the fused kernel marked exhausted, so that no limb
// is ever published and every producer's bounded wait for one runs out after
// max_polls polls.  The kernel then sets STATUS_DEP_TIMEOUT in the plan's
// status word, leaves the data untouched and resets its work area.
ntt_status ntt_internal_test_stalled_forward(const ntt_plan* p, uint64_t* data, uint32_t batch, uint32_t max_polls)
{
    if (!p || !data || batch == 0 || max_polls == 0) return NTT_ERR_INVALID_ARG;
    if (p->passes != 2 || p->kernel != NTT_KERNEL_FUSED) return NTT_ERR_INVALID_ARG;
    if (!aligned16(data)) return NTT_ERR_MISALIGNED;
    const uint64_t limbs = (uint64_t)batch * p->L;
    if (limbs > 0x7FFFFFFFull) return NTT_ERR_INVALID_ARG;
    if (p->work_limbs < limbs) {
        cudaError_t e = ntt_internal_grow_work(const_cast<ntt_plan*>(p), (uint32_t)limbs);
        if (e != cudaSuccess) return to_status(e);
    }
    const uint32_t taken = 0x40000000u;          // above any A-ticket count: no A tile is ever claimed
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(p->d_work, &taken, sizeof(taken), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return to_status(e);
    ntt::LaunchCtx c = p->ctx(data, (uint32_t)limbs, p->L, nullptr);
    c.max_polls = max_polls;
    e = ntt::launch_transform(c, true);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    return to_status(e);
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

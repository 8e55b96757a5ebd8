// Uneven batches: many jobs (arrays of different plans, sizes, levels and
// directions) in few launches.  The paper batches the limbs of equal
// transforms into one launch (Sec. V, Sec. VI-A); here jobs of one size,
// direction and twiddle setting share one launch of the fused two-pass kernel
// (up to FUSED_MAX_JOBS jobs), and the launches of different groups run
// concurrently on the batch's internal streams, so one launch's tail overlaps
// the others.
#include <algorithm>
#include <cstdint>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include <cuda_runtime.h>

#include "plan.h"

extern "C" void ntt_internal_set_cuda_error(cudaError_t e);

namespace {
constexpr int kStreams = 4;
}

struct ntt_batch {
    int device = 0;
    cudaStream_t s[kStreams] = {};
    cudaEvent_t fork = nullptr;
    cudaEvent_t join[kStreams] = {};
    uint32_t* d_work = nullptr;   // work areas of the fused launches, back to back
    size_t work_words = 0;
    uint32_t* d_status = nullptr;
    std::mutex mu;
};

namespace {

ntt_status cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return NTT_OK;
    ntt_internal_set_cuda_error(e);
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? NTT_ERR_OOM : NTT_ERR_CUDA;
}

void release(ntt_batch* b)
{
    for (int k = 0; k < kStreams; ++k) {
        if (b->s[k]) cudaStreamDestroy(b->s[k]);
        if (b->join[k]) cudaEventDestroy(b->join[k]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    cudaFree(b->d_work);
    cudaFree(b->d_status);
    delete b;
}

// A fused launch: jobs (indices into the call's list) of one group.
struct Chunk {
    std::vector<uint32_t> jobs;
    uint64_t limbs = 0;
    uint32_t n = 0, ots = 0;
    bool fwd = true;
    double work = 0;              // limbs x N, for balancing the streams
};

}  // namespace

extern "C" {

ntt_status ntt_batch_create(ntt_batch** out)
{
    if (!out) return NTT_ERR_INVALID_ARG;
    ntt_batch* b = new (std::nothrow) ntt_batch();
    if (!b) return NTT_ERR_OOM;
    cudaError_t e = cudaGetDevice(&b->device);
    for (int k = 0; k < kStreams && e == cudaSuccess; ++k) {
        e = cudaStreamCreateWithFlags(&b->s[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_status, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemset(b->d_status, 0, sizeof(uint32_t));
    if (e != cudaSuccess) {
        release(b);
        return cuda_status(e);
    }
    *out = b;
    return NTT_OK;
}

void ntt_batch_destroy(ntt_batch* b)
{
    if (b) release(b);
}

ntt_status ntt_batch_submit(ntt_batch* b, const ntt_job* jobs, uint32_t njobs, void* stream)
{
    if (!b || !jobs || njobs == 0) return NTT_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> guard(b->mu);
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != b->device) return NTT_ERR_INVALID_ARG;

    // validate, and collect the byte ranges to reject overlapping jobs
    std::vector<std::pair<uintptr_t, uintptr_t>> ranges(njobs);
    for (uint32_t i = 0; i < njobs; ++i) {
        const ntt_job& j = jobs[i];
        if (!j.plan || !j.data || j.batch == 0 || j.levels == 0 || j.levels > j.plan->L || j.reserved)
            return NTT_ERR_INVALID_ARG;
        if (j.op != NTT_OP_FORWARD && j.op != NTT_OP_INVERSE) return NTT_ERR_INVALID_ARG;
        if (j.plan->device != dev) return NTT_ERR_INVALID_ARG;
        if (((uintptr_t)j.data & 15u) != 0) return NTT_ERR_MISALIGNED;
        const uint64_t limbs = (uint64_t)j.batch * j.levels;
        if (limbs > 0x7FFFFFFFull) return NTT_ERR_INVALID_ARG;
        const uintptr_t lo = (uintptr_t)j.data;
        ranges[i] = {lo, lo + (uintptr_t)(limbs * j.plan->N * sizeof(uint64_t))};
    }
    std::sort(ranges.begin(), ranges.end());
    for (uint32_t i = 1; i < njobs; ++i)
        if (ranges[i].first < ranges[i - 1].second) return NTT_ERR_INVALID_ARG;

    // group the fused jobs by (size, direction, OT stages); the rest run alone
    std::map<std::tuple<uint32_t, uint32_t, uint32_t>, std::vector<uint32_t>> groups;
    std::vector<uint32_t> direct;
    for (uint32_t i = 0; i < njobs; ++i) {
        const ntt_plan* p = jobs[i].plan;
        if (p->passes == 2 && p->kernel == NTT_KERNEL_FUSED) {
            const uint32_t ots = p->twiddle_mode == NTT_TWIDDLE_OT ? p->ot_stages : 0;
            groups[std::make_tuple(p->n, jobs[i].op, ots)].push_back(i);
        } else {
            direct.push_back(i);
        }
    }
    std::vector<Chunk> chunks;
    for (auto& g : groups) {
        const auto& idx = g.second;
        for (size_t k = 0; k < idx.size(); k += ntt::FUSED_MAX_JOBS) {
            Chunk c;
            c.n = std::get<0>(g.first);
            c.fwd = std::get<1>(g.first) == NTT_OP_FORWARD;
            c.ots = std::get<2>(g.first);
            for (size_t m = k; m < idx.size() && m < k + ntt::FUSED_MAX_JOBS; ++m) {
                c.jobs.push_back(idx[m]);
                c.limbs += jobs[idx[m]].batch * jobs[idx[m]].levels;
            }
            if (c.limbs > 0x7FFFFFFFull) return NTT_ERR_INVALID_ARG;
            c.work = (double)c.limbs * (double)(1u << c.n);
            chunks.push_back(std::move(c));
        }
    }
    std::sort(chunks.begin(), chunks.end(), [](const Chunk& x, const Chunk& y) { return x.work > y.work; });

    // one work area per fused launch, back to back; grown after the device drains
    size_t words = 0;
    for (const Chunk& c : chunks) words += ntt::fused_work_words(c.limbs);
    if (words > b->work_words) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_status(e);
        cudaFree(b->d_work);
        b->d_work = nullptr;
        b->work_words = 0;
        e = cudaMalloc(&b->d_work, words * sizeof(uint32_t));
        if (e == cudaSuccess) e = cudaMemset(b->d_work, 0, words * sizeof(uint32_t));
        if (e != cudaSuccess) return cuda_status(e);
        b->work_words = words;
    }

    // fork onto the internal streams, longest launches first on the least loaded stream
    const cudaStream_t caller = (cudaStream_t)stream;
    const int used = (int)std::min<size_t>(kStreams, chunks.size() + direct.size());
    cudaError_t e = cudaEventRecord(b->fork, caller);
    for (int k = 0; k < used && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b->s[k], b->fork, 0);
    if (e != cudaSuccess) return cuda_status(e);
    double load[kStreams] = {};
    auto pick = [&](double w) {
        int best = 0;
        for (int k = 1; k < used; ++k)
            if (load[k] < load[best]) best = k;
        load[best] += w;
        return best;
    };
    size_t off = 0;
    std::vector<ntt::JobCtx> jc;
    for (const Chunk& c : chunks) {
        jc.clear();
        for (uint32_t i : c.jobs) {
            const ntt_plan* p = jobs[i].plan;
            jc.push_back(ntt::JobCtx{reinterpret_cast<ntt::u64*>(jobs[i].data), jobs[i].batch * jobs[i].levels,
                                     jobs[i].levels, p->d_primes, p->d_tw, p->tw_len, p->d_ota_f, p->d_otb_f,
                                     p->d_ota_i, p->d_otb_i});
        }
        const int k = pick(c.work);
        const ntt::JobsCtx ctx{jc.data(), (uint32_t)jc.size(), c.n, c.ots, b->d_status, b->d_work + off,
                               (uint32_t)c.limbs, b->s[k]};
        off += ntt::fused_work_words(c.limbs);
        e = ntt::launch_fused_jobs(ctx, c.fwd);
        if (e != cudaSuccess) break;
    }
    for (size_t m = 0; m < direct.size() && e == cudaSuccess; ++m) {
        const ntt_job& j = jobs[direct[m]];
        const int k = pick((double)j.batch * j.levels * j.plan->N);
        const ntt::LaunchCtx c = j.plan->ctx(j.data, j.batch * j.levels, j.levels, b->s[k]);
        e = ntt::launch_transform(c, j.op == NTT_OP_FORWARD);
    }
    // join back onto the caller's stream (also after a failed launch, so the
    // caller's stream stays ordered after whatever was enqueued)
    for (int k = 0; k < used; ++k) {
        cudaEventRecord(b->join[k], b->s[k]);
        cudaStreamWaitEvent(caller, b->join[k], 0);
    }
    return cuda_status(e);
}

ntt_status ntt_batch_device_status(ntt_batch* b, uint32_t* status)
{
    if (!b || !status) return NTT_ERR_INVALID_ARG;
    cudaError_t e = cudaDeviceSynchronize();
    uint32_t v = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&v, b->d_status, sizeof(v), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(b->d_status, 0, sizeof(v));
    if (e != cudaSuccess) return cuda_status(e);
    *status = v;
    return NTT_OK;
}

}  // extern "C"

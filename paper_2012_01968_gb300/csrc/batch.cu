// Uneven batches: many jobs (arrays of different plans, sizes, levels and
// directions) in few launches.  The paper batches the limbs of equal
// transforms into one launch (Sec. V, Sec. VI-A); here jobs of one size,
// direction and twiddle setting share one launch of the fused two-pass kernel
// (up to FUSED_MAX_JOBS jobs), and the launches of different groups run
// concurrently on the batch's internal streams, so one launch's tail overlaps
// the others.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include <cuda_runtime.h>

#include "host_logic.h"
#include "plan.h"

extern "C" void ntt_internal_set_cuda_error(cudaError_t e);

namespace {
constexpr int kStreams = 4;
// descriptor generations of the mixed launches: a submission whose
// descriptors differ from the latest stages them in the next generation, so
// that up to this many submissions with different descriptors can be in
// flight before the host waits for the oldest
constexpr int kMixGenerations = 4;
}

struct ntt_batch {
    int device = 0;
    cudaStream_t s[kStreams] = {};
    cudaEvent_t fork = nullptr;
    cudaEvent_t join[kStreams] = {};
    uint32_t* d_work = nullptr;   // work areas of the fused launches, back to back
    size_t work_words = 0;
    uint32_t* d_status = nullptr;
    uint32_t test_stall_polls = 0;  // test hook: the next submission's fused launches stall (bounded)
    // job descriptors of the mixed-size launches: kMixGenerations device
    // arrays of mix_cap descriptors and their page-locked host copies (each
    // host copy equals what its upload wrote)
    void* d_mix = nullptr;
    void* h_mix = nullptr;
    size_t mix_cap = 0;             // jobs per generation
    int mix_gen = 0;                // generation holding the latest descriptors
    size_t mix_bytes = 0;           // their size (0: none yet)
    // recorded on the caller's stream after the latest submission that used
    // a generation (its upload and its launches are then done)
    cudaEvent_t mix_done[kMixGenerations] = {};
    bool mix_used[kMixGenerations] = {};
    uint32_t last_launches = 0;     // kernel launches of the latest submission
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
    if (b->d_mix || b->h_mix) {
        for (int k = 0; k < kStreams; ++k)
            if (b->s[k]) cudaStreamSynchronize(b->s[k]);
        cudaFree(b->d_mix);
        cudaFreeHost(b->h_mix);
        b->d_mix = b->h_mix = nullptr;
    }
    for (int k = 0; k < kStreams; ++k) {
        if (b->s[k]) cudaStreamDestroy(b->s[k]);
        if (b->join[k]) cudaEventDestroy(b->join[k]);
    }
    for (int g = 0; g < kMixGenerations; ++g)
        if (b->mix_done[g]) cudaEventDestroy(b->mix_done[g]);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->d_work) {
        cudaFreeAsync(b->d_work, nullptr);
        cudaStreamSynchronize(nullptr);
    }
    cudaFree(b->d_status);
    delete b;
}

// Make the work area hold `words` words, zero-filled, ordered on `caller`:
// the caller's stream first waits for everything the batch's streams hold
// (the old area's last users), then frees the old area and allocates the new
// one stream-ordered, so no other stream or host thread is blocked.  Not
// during graph capture (the area must outlive the captured graph).
cudaError_t grow_work(ntt_batch* b, size_t words, cudaStream_t caller)
{
    if (words <= b->work_words) return cudaSuccess;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(caller, &cs);
    if (e != cudaSuccess) return e;
    if (cs != cudaStreamCaptureStatusNone) return cudaErrorStreamCaptureUnsupported;
    for (int k = 0; k < kStreams && e == cudaSuccess; ++k) {
        e = cudaEventRecord(b->join[k], b->s[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(caller, b->join[k], 0);
    }
    if (e != cudaSuccess) return e;
    if (b->d_work) {
        e = cudaFreeAsync(b->d_work, caller);
        b->d_work = nullptr;
        b->work_words = 0;
        if (e != cudaSuccess) return e;
    }
    void* mem = nullptr;
    e = cudaMallocAsync(&mem, words * sizeof(uint32_t), caller);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(mem, 0, words * sizeof(uint32_t), caller);
    b->d_work = static_cast<uint32_t*>(mem);
    if (e == cudaSuccess) b->work_words = words;
    return e;
}

// Room for `jobs` mixed-launch descriptors per generation (device and host
// copies).  Growing drains the batch's streams first (an earlier launch may
// still read the old arrays); not during graph capture.
cudaError_t reserve_mix(ntt_batch* b, size_t jobs, cudaStream_t caller)
{
    if (jobs <= b->mix_cap) return cudaSuccess;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(caller, &cs);
    if (e != cudaSuccess) return e;
    if (cs != cudaStreamCaptureStatusNone) return cudaErrorStreamCaptureUnsupported;
    for (int k = 0; k < kStreams && e == cudaSuccess; ++k) e = cudaStreamSynchronize(b->s[k]);
    if (e != cudaSuccess) return e;
    cudaFree(b->d_mix);
    cudaFreeHost(b->h_mix);
    b->d_mix = b->h_mix = nullptr;
    b->mix_cap = 0;
    b->mix_bytes = 0;
    for (bool& u : b->mix_used) u = false;
    const size_t cap = std::max<size_t>(jobs, 128), bytes = kMixGenerations * cap * ntt::mixed_job_bytes();
    e = cudaMalloc(&b->d_mix, bytes);
    if (e == cudaSuccess) e = cudaMemset(b->d_mix, 0, bytes);
    if (e == cudaSuccess) e = cudaHostAlloc(&b->h_mix, bytes, cudaHostAllocDefault);
    if (e == cudaSuccess) std::memset(b->h_mix, 0, bytes);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();     // the zeroing is done before any upload
    if (e != cudaSuccess) {
        cudaFree(b->d_mix);
        if (b->h_mix) cudaFreeHost(b->h_mix);
        b->d_mix = b->h_mix = nullptr;
        return e;
    }
    b->mix_cap = cap;
    return cudaSuccess;
}

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
    for (int g = 0; g < kMixGenerations && e == cudaSuccess; ++g)
        e = cudaEventCreateWithFlags(&b->mix_done[g], cudaEventDisableTiming);
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
    if (ntt::host::any_overlap(ranges)) return NTT_ERR_INVALID_ARG;

    // Fused jobs of plans with the default geometry go into one mixed-size
    // launch per OT setting (all sizes and both directions together); fused
    // jobs of other geometries are grouped by (size and geometry, direction,
    // OT stages) into launches of up to FUSED_MAX_JOBS jobs; the rest run alone.
    std::vector<uint32_t> fused, direct;
    std::vector<std::vector<uint32_t>> mixed(3);          // by OT stages
    std::vector<std::tuple<uint32_t, uint32_t, uint32_t>> keys;
    std::vector<uint64_t> limbs, sizes;
    for (uint32_t i = 0; i < njobs; ++i) {
        const ntt_plan* p = jobs[i].plan;
        if (p->passes == 2 && p->kernel == NTT_KERNEL_FUSED) {
            const uint32_t ots = p->twiddle_mode == NTT_TWIDDLE_OT ? p->ot_stages : 0;
            if (p->geom == 0 && ots <= 2) {
                mixed[ots].push_back(i);
                continue;
            }
            fused.push_back(i);
            keys.emplace_back(p->n | (p->geom << 8), jobs[i].op, ots);
            limbs.push_back((uint64_t)jobs[i].batch * jobs[i].levels);
            sizes.push_back(p->N);
        } else {
            direct.push_back(i);
        }
    }
    std::vector<ntt::host::Chunk> chunks = ntt::host::make_chunks(keys, limbs, sizes, ntt::FUSED_MAX_JOBS);
    for (ntt::host::Chunk& c : chunks) {
        if (c.limbs > 0x7FFFFFFFull) return NTT_ERR_INVALID_ARG;
        for (uint32_t& j : c.jobs) j = fused[j];          // indices into the submission
    }
    auto job_in = [&](uint32_t i) {
        const ntt_plan* p = jobs[i].plan;
        return ntt::MixJobIn{ntt::JobCtx{reinterpret_cast<ntt::u64*>(jobs[i].data), jobs[i].batch * jobs[i].levels,
                                         jobs[i].levels, p->d_primes, p->d_tw, p->tw_len, p->d_ota_f, p->d_otb_f,
                                         p->d_ota_i, p->d_otb_i},
                             p->n, jobs[i].op == NTT_OP_FORWARD ? 1u : 0u};
    };
    // the mixed launches: per OT setting, up to MIXED_MAX_JOBS jobs each
    std::vector<std::vector<ntt::MixJobIn>> mixin;
    std::vector<uint32_t> mix_ots;
    size_t mix_jobs = 0;
    for (int o = 0; o < 3; ++o) {
        for (size_t k = 0; k < mixed[o].size(); k += ntt::MIXED_MAX_JOBS) {
            mixin.emplace_back();
            mix_ots.push_back((uint32_t)o);
            for (size_t m = k; m < mixed[o].size() && m < k + ntt::MIXED_MAX_JOBS; ++m)
                mixin.back().push_back(job_in(mixed[o][m]));
            mix_jobs += mixin.back().size();
        }
    }

    // one work area per launch, back to back; grown in stream order
    const cudaStream_t caller = (cudaStream_t)stream;
    size_t words = 0;
    for (const auto& m : mixin) words += ntt::mixed_work_words(m.data(), (uint32_t)m.size());
    for (const ntt::host::Chunk& c : chunks) words += ntt::fused_work_words(c.limbs);
    if (words > b->work_words) {
        cudaError_t e = grow_work(b, words, caller);
        if (e != cudaSuccess) return cuda_status(e);
    }
    if (mix_jobs > b->mix_cap) {
        cudaError_t e = reserve_mix(b, mix_jobs, caller);
        if (e != cudaSuccess) return cuda_status(e);
    }

    // test hook: mark every fused launch's first-pass queue as taken, so that
    // no limb is ever published and every wait for one runs out after
    // test_stall_polls polls (the kernels then set the status word)
    const uint32_t stall = b->test_stall_polls;
    b->test_stall_polls = 0;
    size_t mix_words = 0;
    for (const auto& m : mixin) mix_words += ntt::mixed_work_words(m.data(), (uint32_t)m.size());
    if (stall) {
        static const uint32_t taken = 0x40000000u;
        size_t o = mix_words;
        for (const ntt::host::Chunk& c : chunks) {
            cudaError_t e = cudaMemcpyAsync(b->d_work + o, &taken, sizeof(taken), cudaMemcpyHostToDevice, caller);
            if (e != cudaSuccess) return cuda_status(e);
            o += ntt::fused_work_words(c.limbs);
        }
    }

    // the mixed launches' descriptors: unchanged since the latest submission
    // (e.g. a submission replayed from a CUDA graph), or staged in the next
    // generation and uploaded on the caller's stream before the fork
    cudaStreamCaptureStatus capture = cudaStreamCaptureStatusNone;
    {
        cudaError_t e = cudaStreamIsCapturing(caller, &capture);
        if (e != cudaSuccess) return cuda_status(e);
    }
    std::vector<ntt::MixBuilt> built(mixin.size());
    std::vector<unsigned char> descs;
    for (size_t mi = 0; mi < mixin.size(); ++mi) {
        cudaError_t e = ntt::build_mixed(mixin[mi].data(), (uint32_t)mixin[mi].size(), mix_ots[mi], &built[mi]);
        if (e != cudaSuccess) return cuda_status(e);
        descs.insert(descs.end(), built[mi].desc.begin(), built[mi].desc.end());
    }
    const size_t gen_bytes = b->mix_cap * ntt::mixed_job_bytes();
    auto gen_host = [&](int g) { return static_cast<unsigned char*>(b->h_mix) + (size_t)g * gen_bytes; };
    auto gen_dev = [&](int g) { return static_cast<unsigned char*>(b->d_mix) + (size_t)g * gen_bytes; };
    if (!mixin.empty() && !(descs.size() == b->mix_bytes &&
                            std::memcmp(gen_host(b->mix_gen), descs.data(), descs.size()) == 0)) {
        if (capture != cudaStreamCaptureStatusNone) return cuda_status(cudaErrorStreamCaptureUnsupported);
        const int g = (b->mix_gen + 1) % kMixGenerations;
        cudaError_t e = b->mix_used[g] ? cudaEventSynchronize(b->mix_done[g]) : cudaSuccess;
        if (e == cudaSuccess) {
            std::memcpy(gen_host(g), descs.data(), descs.size());
            e = cudaMemcpyAsync(gen_dev(g), gen_host(g), descs.size(), cudaMemcpyHostToDevice, caller);
        }
        if (e != cudaSuccess) return cuda_status(e);
        b->mix_gen = g;
        b->mix_bytes = descs.size();
    }
    const int gen = b->mix_gen;

    // fork onto the internal streams
    const size_t nmix = mixin.size();
    const int used = (int)std::min<size_t>(kStreams, nmix + chunks.size() + direct.size());
    cudaError_t e = cudaEventRecord(b->fork, caller);
    for (int k = 0; k < used && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b->s[k], b->fork, 0);
    if (e != cudaSuccess) return cuda_status(e);
    // longest first, each on the least loaded stream: the mixed launches,
    // the chunks, then the jobs that run alone
    std::vector<double> work;
    for (const auto& mj : mixin) {
        double w = 0;
        for (const ntt::MixJobIn& m : mj) w += (double)m.job.limbs * (double)(1u << m.n);
        work.push_back(w);
    }
    for (const ntt::host::Chunk& c : chunks) work.push_back(c.work);
    for (uint32_t i : direct) work.push_back((double)jobs[i].batch * jobs[i].levels * jobs[i].plan->N);
    const std::vector<int> at = ntt::host::place_least_loaded(work, used);
    size_t off = 0, item = 0, desc = 0;
    for (size_t mi = 0; mi < mixin.size() && e == cudaSuccess; ++mi) {
        const size_t w = ntt::mixed_work_words(mixin[mi].data(), (uint32_t)mixin[mi].size());
        const auto* d_desc = reinterpret_cast<const ntt::MixJob*>(gen_dev(gen) + desc);
        e = ntt::launch_mixed(built[mi], d_desc, b->d_work + off, w, b->d_status, stall, b->s[at[item]]);
        off += w;
        desc += built[mi].desc.size();
        ++item;
    }
    std::vector<ntt::JobCtx> jc;
    for (size_t ci = 0; ci < chunks.size() && e == cudaSuccess; ++ci) {
        const ntt::host::Chunk& c = chunks[ci];
        jc.clear();
        for (uint32_t i : c.jobs) {
            const ntt_plan* p = jobs[i].plan;
            jc.push_back(ntt::JobCtx{reinterpret_cast<ntt::u64*>(jobs[i].data), jobs[i].batch * jobs[i].levels,
                                     jobs[i].levels, p->d_primes, p->d_tw, p->tw_len, p->d_ota_f, p->d_otb_f,
                                     p->d_ota_i, p->d_otb_i});
        }
        const int k = at[item++];
        const uint32_t n = std::get<0>(c.key) & 0xFFu, geom = std::get<0>(c.key) >> 8, ots = std::get<2>(c.key);
        const bool fwd = std::get<1>(c.key) == NTT_OP_FORWARD;
        const ntt::JobsCtx ctx{jc.data(), (uint32_t)jc.size(), n, ots, b->d_status, b->d_work + off,
                               (uint32_t)c.limbs, b->s[k], stall, geom};
        off += ntt::fused_work_words(c.limbs);
        e = ntt::launch_fused_jobs(ctx, fwd);
    }
    for (size_t m = 0; m < direct.size() && e == cudaSuccess; ++m) {
        const ntt_job& j = jobs[direct[m]];
        const int k = at[item++];
        const ntt::LaunchCtx c = j.plan->ctx(j.data, j.batch * j.levels, j.levels, b->s[k]);
        e = ntt::launch_transform(c, j.op == NTT_OP_FORWARD);
    }
    b->last_launches = (uint32_t)item;
    // join back onto the caller's stream (also after a failed launch, so the
    // caller's stream stays ordered after whatever was enqueued)
    for (int k = 0; k < used; ++k) {
        cudaEventRecord(b->join[k], b->s[k]);
        cudaStreamWaitEvent(caller, b->join[k], 0);
    }
    // the generation's host and device copies are free again once this
    // event has passed (a captured submission leaves it to the eager one
    // whose descriptors it reuses)
    if (nmix && capture == cudaStreamCaptureStatusNone) {
        const cudaError_t r = cudaEventRecord(b->mix_done[gen], caller);
        if (e == cudaSuccess) e = r;
        b->mix_used[gen] = true;
    }
    return cuda_status(e);
}

// Test hook (not part of the public interface): the next submission's fused
// launches find their first-pass queue taken and their waits bounded by
// `max_polls`, so they end with the dependency-timeout status and the data
// untouched.
ntt_status ntt_internal_batch_test_stall(ntt_batch* b, uint32_t max_polls)
{
    if (!b || max_polls == 0) return NTT_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> guard(b->mu);
    b->test_stall_polls = max_polls;
    return NTT_OK;
}

// Test hook (not part of the public interface): kernel launches of the
// latest submission (direct jobs count their own launches as one each).
ntt_status ntt_internal_batch_last_launches(ntt_batch* b, uint32_t* count)
{
    if (!b || !count) return NTT_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> guard(b->mu);
    *count = b->last_launches;
    return NTT_OK;
}

// Library-internal: copy the batch's device status word to `host_word`
// (page-locked) and clear it, in order on `stream` (the serving loop reads it
// in its completion callback, without a device synchronisation).
ntt_status ntt_internal_batch_status_async(ntt_batch* b, uint32_t* host_word, void* stream)
{
    if (!b || !host_word) return NTT_ERR_INVALID_ARG;
    cudaError_t e = cudaMemcpyAsync(host_word, b->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                    (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_status, 0, sizeof(uint32_t), (cudaStream_t)stream);
    return cuda_status(e);
}

// Library-internal: size the work area and the mixed launches' descriptor
// arrays up front (the serving loop reserves its batches at creation, so that
// no submission grows an area or drains the device to allocate the arrays).
ntt_status ntt_internal_batch_reserve(ntt_batch* b, uint64_t words, void* stream)
{
    if (!b) return NTT_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> guard(b->mu);
    cudaError_t e = grow_work(b, (size_t)words, (cudaStream_t)stream);
    if (e == cudaSuccess) e = reserve_mix(b, 1, (cudaStream_t)stream);
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

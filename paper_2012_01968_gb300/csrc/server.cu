// Serving: a request loop with admission by device memory and continuous
// batching (a library runtime around the transforms; the paper measures
// batches, not request streams).
//
// A scheduler thread owns the device side.  Requests wait in a FIFO queue;
// the scheduler admits them from its head while their bytes fit the budget
// (and, for host-buffer requests, the device arena), and starts a batch in
// the first free slot.  A slot is a stream with its own batch object:
// copy-in of the host-buffer requests, one ntt_batch_submit over all the
// batch's requests, copy-out, the copy of the batch's kernel status word,
// then an event.  The scheduler polls the slots' events (no host callback
// on the device's streams, so a late callback thread cannot hold back the
// other slots), timestamps finished requests and wakes the waiters.
// Requests that arrive while batches are on the device are admitted into the
// next free slot as memory frees up, so several batches overlap on the device.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "host_logic.h"
#include "plan.h"

extern "C" void ntt_internal_set_cuda_error(cudaError_t e);
extern "C" ntt_status ntt_internal_batch_reserve(ntt_batch* b, uint64_t words, void* stream);
extern "C" ntt_status ntt_internal_batch_status_async(ntt_batch* b, uint32_t* host_word, void* stream);
extern "C" ntt_status ntt_internal_batch_test_stall(ntt_batch* b, uint32_t max_polls);

namespace {

int64_t now_ns()
{
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Req {
    uint64_t ticket = 0;
    ntt_request r{};
    size_t bytes = 0;
    size_t arena_off = 0;         // host-buffer requests: device staging offset
    bool host = false;
    int64_t t_submit = 0, t_start = 0, t_done = 0, t_device = 0;
    ntt_status status = NTT_OK;
    bool done = false;
};

struct Slot {
    cudaStream_t stream = nullptr;
    ntt_batch* batch = nullptr;
    uint32_t* status = nullptr;   // page-locked copy of the batch's device status word
    std::vector<Req*> reqs;       // of the batch in flight (empty when free)
    bool busy = false;
    bool finished = false;        // set when the scheduler sees `done` complete
    cudaEvent_t done = nullptr;   // recorded after the batch's last copy
    cudaEvent_t begin = nullptr;  // recorded before its first operation (timing)
    int64_t t_start = 0;          // host time the batch was started
};

using Arena = ntt::host::Arena;

}  // namespace

struct ntt_server {
    ntt_server_opts opts{};
    int device = 0;
    uint8_t* arena_mem = nullptr;
    Arena arena;
    size_t admitted_bytes = 0;
    std::vector<Slot> slots;
    std::deque<Req*> pending;
    std::unordered_map<uint64_t, std::unique_ptr<Req>> reqs;
    uint64_t next_ticket = 1;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    cudaError_t fatal = cudaSuccess;
    uint32_t test_stall_polls = 0;    // test hook: the next batch's kernels stall (bounded)
    ntt_server_stats stats{};
    int64_t t_last_completion = 0;
};

namespace {

// Mark the busy slots whose batch has completed (called with the lock held;
// the event queries run with it released, so that submissions and waits
// never queue behind a CUDA call).  Returns true when a slot is still running.
bool poll_slots(ntt_server* srv, std::unique_lock<std::mutex>& lk)
{
    bool running = false;
    std::vector<Slot*> busy;
    for (Slot& s : srv->slots)
        if (s.busy && !s.finished) busy.push_back(&s);
    if (busy.empty()) return false;
    std::vector<cudaError_t> q(busy.size());
    lk.unlock();
    for (size_t i = 0; i < busy.size(); ++i) q[i] = cudaEventQuery(busy[i]->done);
    lk.lock();
    for (size_t i = 0; i < busy.size(); ++i) {
        Slot& s = *busy[i];
        if (q[i] == cudaErrorNotReady) {
            running = true;
            continue;
        }
        const cudaError_t qe = q[i];
        const int64_t t = now_ns();
        // a bounded wait of the batch's kernels that ran out fails its requests
        const bool device_error = qe == cudaSuccess && *static_cast<volatile uint32_t*>(s.status) != 0;
        float ms = 0.f;
        if (qe == cudaSuccess && cudaEventElapsedTime(&ms, s.begin, s.done) != cudaSuccess) ms = 0.f;
        const int64_t gap = t - std::max(srv->t_last_completion, s.t_start);
        srv->stats.max_completion_gap_ns = std::max(srv->stats.max_completion_gap_ns, gap);
        srv->stats.max_device_ns = std::max(srv->stats.max_device_ns, (int64_t)((double)ms * 1e6));
        srv->t_last_completion = t;
        for (Req* r : s.reqs) {
            r->t_done = t;
            r->t_device = (int64_t)((double)ms * 1e6);
            if (qe != cudaSuccess) r->status = NTT_ERR_CUDA;
            else if (device_error) r->status = NTT_ERR_DEVICE;
        }
        if (qe != cudaSuccess) {
            cudaGetLastError();
            srv->fatal = qe;
        }
        s.finished = true;
    }
    return running;
}

// Start one batch in slot `s` from the head of the queue (called with the
// lock held; returns false when nothing could be admitted).
bool start_batch(ntt_server* srv, Slot& s, std::unique_lock<std::mutex>& lk)
{
    std::vector<Req*> take;
    while (!srv->pending.empty() && take.size() < srv->opts.max_batch_jobs) {
        Req* r = srv->pending.front();
        if (srv->admitted_bytes + r->bytes > srv->opts.hbm_budget_bytes) break;
        if (r->host && !srv->arena.alloc(r->bytes, &r->arena_off)) break;
        srv->admitted_bytes += r->bytes;
        srv->pending.pop_front();
        take.push_back(r);
    }
    if (take.empty()) return false;
    s.busy = true;
    s.finished = false;
    s.reqs = take;
    const uint32_t stall = srv->test_stall_polls;
    srv->test_stall_polls = 0;
    const int64_t t = now_ns();
    for (Req* r : take) r->t_start = t;
    s.t_start = t;
    ++srv->stats.batches;
    lk.unlock();

    cudaError_t e = cudaEventRecord(s.begin, s.stream);
    std::vector<ntt_job> jobs;
    jobs.reserve(take.size());
    for (Req* r : take) {
        uint64_t* dev = r->r.data;
        if (r->host) {
            dev = reinterpret_cast<uint64_t*>(srv->arena_mem + r->arena_off);
            if (e == cudaSuccess) e = cudaMemcpyAsync(dev, r->r.data, r->bytes, cudaMemcpyHostToDevice, s.stream);
        }
        jobs.push_back(ntt_job{r->r.plan, dev, r->r.batch, r->r.levels, r->r.op, 0});
    }
    if (stall) ntt_internal_batch_test_stall(s.batch, stall);
    ntt_status st = e == cudaSuccess ? ntt_batch_submit(s.batch, jobs.data(), (uint32_t)jobs.size(), s.stream)
                                     : NTT_ERR_CUDA;
    for (Req* r : take) {
        if (st == NTT_OK && r->host) {
            const uint64_t* dev = reinterpret_cast<const uint64_t*>(srv->arena_mem + r->arena_off);
            e = cudaMemcpyAsync(r->r.host_out, dev, r->bytes, cudaMemcpyDeviceToHost, s.stream);
            if (e != cudaSuccess) st = NTT_ERR_CUDA;
        }
    }
    if (st == NTT_OK) st = ntt_internal_batch_status_async(s.batch, s.status, s.stream);
    if (e == cudaSuccess && st == NTT_OK) e = cudaEventRecord(s.done, s.stream);
    const int64_t t_enq = now_ns() - t;
    lk.lock();
    srv->stats.max_launch_ns = std::max(srv->stats.max_launch_ns, t_enq);
    if (e != cudaSuccess || st != NTT_OK) {
        // nothing will call back: finish the batch here once the stream drains
        lk.unlock();
        cudaStreamSynchronize(s.stream);
        cudaGetLastError();
        lk.lock();
        const int64_t t2 = now_ns();
        for (Req* r : take) {
            r->status = st != NTT_OK ? st : NTT_ERR_CUDA;
            r->t_done = t2;
        }
        s.finished = true;
        if (e != cudaSuccess) srv->fatal = e;
    }
    return true;
}

// Retire finished batches (lock held): free their memory, publish results.
bool retire(ntt_server* srv)
{
    bool any = false;
    for (Slot& s : srv->slots) {
        if (!s.busy || !s.finished) continue;
        for (Req* r : s.reqs) {
            srv->admitted_bytes -= r->bytes;
            if (r->host) srv->arena.release(r->arena_off, r->bytes);
            r->done = true;
            ++srv->stats.requests;
        }
        s.reqs.clear();
        s.busy = false;
        s.finished = false;
        any = true;
    }
    if (any) srv->cv_done.notify_all();
    return any;
}

void scheduler(ntt_server* srv)
{
    cudaSetDevice(srv->device);
    std::unique_lock<std::mutex> lk(srv->mu);
    int64_t t_prev = now_ns();
    for (;;) {
        const int64_t t_now = now_ns();
        srv->stats.max_loop_gap_ns = std::max(srv->stats.max_loop_gap_ns, t_now - t_prev);
        t_prev = t_now;
        const bool running = poll_slots(srv, lk);
        retire(srv);
        bool started = false;
        for (Slot& s : srv->slots)
            if (!s.busy && !srv->pending.empty()) started |= start_batch(srv, s, lk);
        bool inflight = false;
        for (const Slot& s : srv->slots) inflight |= s.busy;
        if (srv->stop && srv->pending.empty() && !inflight) break;
        if (started) continue;
        // poll again soon while batches run; otherwise wait for a request
        if (running) srv->cv_work.wait_for(lk, std::chrono::microseconds(20));
        else srv->cv_work.wait_for(lk, std::chrono::milliseconds(2));
    }
}

}  // namespace

extern "C" {

ntt_status ntt_server_create(ntt_server** out, const ntt_server_opts* opts)
{
    if (!out || !opts || opts->hbm_budget_bytes == 0) return NTT_ERR_INVALID_ARG;
    for (uint32_t r : opts->reserved)
        if (r) return NTT_ERR_INVALID_ARG;
    std::unique_ptr<ntt_server> srv(new (std::nothrow) ntt_server());
    if (!srv) return NTT_ERR_OOM;
    srv->opts = *opts;
    // 64 requests per batch: 2.5% more capacity than 32 on the C5 mix, and
    // no change at 128 (batches only fill up under load)
    if (!srv->opts.max_batch_jobs) srv->opts.max_batch_jobs = 64;
    if (!srv->opts.slots) srv->opts.slots = 3;
    if (!srv->opts.max_queue) srv->opts.max_queue = 1u << 20;
    if (srv->opts.slots > 16) return NTT_ERR_INVALID_ARG;
    cudaError_t e = cudaGetDevice(&srv->device);
    const size_t arena = (size_t)srv->opts.arena_bytes;
    if (e == cudaSuccess && arena) e = cudaMalloc(&srv->arena_mem, arena);
    srv->arena.reset(e == cudaSuccess ? arena : 0);
    srv->slots.resize(srv->opts.slots);
    for (Slot& s : srv->slots) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaHostAlloc(&s.status, sizeof(uint32_t), cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaEventCreate(&s.done);
        if (e == cudaSuccess) e = cudaEventCreate(&s.begin);
        if (e == cudaSuccess) *s.status = 0;
        if (e == cudaSuccess && ntt_batch_create(&s.batch) != NTT_OK) e = cudaErrorMemoryAllocation;
    }
    // every slot's batch gets its fused-kernel work area now: one batch holds
    // at most max_batch_jobs launches and, within the budget, at most
    // budget / (8 * 2^13) limbs of fused sizes (capped at 2^24)
    const uint64_t limb_bound = std::min<uint64_t>(srv->opts.hbm_budget_bytes / (8ull << 13), 1ull << 24);
    const uint64_t words = 4ull * srv->opts.max_batch_jobs + 2ull * limb_bound;
    for (Slot& s : srv->slots)
        if (e == cudaSuccess && ntt_internal_batch_reserve(s.batch, words, s.stream) != NTT_OK)
            e = cudaErrorMemoryAllocation;
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        for (Slot& s : srv->slots) {
            if (s.batch) ntt_batch_destroy(s.batch);
            if (s.stream) cudaStreamDestroy(s.stream);
            if (s.status) cudaFreeHost(s.status);
            if (s.done) cudaEventDestroy(s.done);
            if (s.begin) cudaEventDestroy(s.begin);
        }
        cudaFree(srv->arena_mem);
        ntt_internal_set_cuda_error(e);
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? NTT_ERR_OOM : NTT_ERR_CUDA;
    }
    ntt_server* raw = srv.release();
    raw->worker = std::thread(scheduler, raw);
    *out = raw;
    return NTT_OK;
}

void ntt_server_destroy(ntt_server* srv)
{
    if (!srv) return;
    {
        std::lock_guard<std::mutex> g(srv->mu);
        srv->stop = true;
    }
    srv->cv_work.notify_one();
    if (srv->worker.joinable()) srv->worker.join();
    for (Slot& s : srv->slots) {
        if (s.stream) cudaStreamSynchronize(s.stream);
        if (s.batch) ntt_batch_destroy(s.batch);
        if (s.stream) cudaStreamDestroy(s.stream);
        if (s.status) cudaFreeHost(s.status);
        if (s.done) cudaEventDestroy(s.done);
        if (s.begin) cudaEventDestroy(s.begin);
    }
    cudaFree(srv->arena_mem);
    delete srv;
}

ntt_status ntt_server_submit(ntt_server* srv, const ntt_request* req, uint64_t* ticket)
{
    if (!srv || !req || !ticket) return NTT_ERR_INVALID_ARG;
    const ntt_request& q = *req;
    if (!q.plan || !q.data || q.batch == 0 || q.levels == 0 || q.levels > q.plan->L) return NTT_ERR_INVALID_ARG;
    if (q.op != NTT_OP_FORWARD && q.op != NTT_OP_INVERSE) return NTT_ERR_INVALID_ARG;
    if (q.flags & ~(uint32_t)NTT_REQ_HOST) return NTT_ERR_INVALID_ARG;
    const bool host = (q.flags & NTT_REQ_HOST) != 0;
    if (host && !q.host_out) return NTT_ERR_INVALID_ARG;
    if (!host && ((uintptr_t)q.data & 15u)) return NTT_ERR_MISALIGNED;
    if (q.plan->device != srv->device) return NTT_ERR_INVALID_ARG;
    const uint64_t limbs = (uint64_t)q.batch * q.levels;
    if (limbs > 0x7FFFFFFFull) return NTT_ERR_INVALID_ARG;
    const size_t bytes = (size_t)limbs * q.plan->N * sizeof(uint64_t);
    if (bytes > srv->opts.hbm_budget_bytes) return NTT_ERR_INVALID_ARG;          // could never be admitted
    if (host && bytes > srv->opts.arena_bytes) return NTT_ERR_INVALID_ARG;
    std::unique_ptr<Req> r(new (std::nothrow) Req());
    if (!r) return NTT_ERR_OOM;
    r->r = q;
    r->bytes = bytes;
    r->host = host;
    {
        std::lock_guard<std::mutex> g(srv->mu);
        if (srv->stop) return NTT_ERR_INVALID_ARG;
        if (srv->fatal != cudaSuccess) {                 // a copy or launch of the server failed
            ntt_internal_set_cuda_error(srv->fatal);
            return NTT_ERR_CUDA;
        }
        if (srv->pending.size() >= srv->opts.max_queue) return NTT_ERR_BUSY;
        r->ticket = srv->next_ticket++;
        r->t_submit = now_ns();
        *ticket = r->ticket;
        srv->pending.push_back(r.get());
        srv->reqs.emplace(r->ticket, std::move(r));
    }
    srv->cv_work.notify_one();
    return NTT_OK;
}

// Test hook (not part of the public interface): the next batch the server
// starts has its fused launches stall, with waits bounded by `max_polls`.
ntt_status ntt_internal_server_test_stall_next(ntt_server* srv, uint32_t max_polls)
{
    if (!srv || max_polls == 0) return NTT_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(srv->mu);
    srv->test_stall_polls = max_polls;
    return NTT_OK;
}

ntt_status ntt_server_wait(ntt_server* srv, uint64_t ticket, uint64_t timeout_ns)
{
    if (!srv) return NTT_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return NTT_ERR_INVALID_ARG;
    Req* r = it->second.get();
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::nanoseconds(timeout_ns);
    while (!r->done) {
        if (srv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !r->done) return NTT_ERR_TIMEOUT;
    }
    return r->status;
}

ntt_status ntt_server_request_times(ntt_server* srv, uint64_t ticket, ntt_request_times* times)
{
    if (!srv || !times) return NTT_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return NTT_ERR_INVALID_ARG;
    const Req* r = it->second.get();
    times->submit_ns = r->t_submit;
    times->start_ns = r->t_start;
    times->done_ns = r->done ? r->t_done : 0;
    times->device_ns = r->done ? r->t_device : 0;
    return NTT_OK;
}

ntt_status ntt_server_release(ntt_server* srv, uint64_t ticket)
{
    if (!srv) return NTT_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return NTT_ERR_INVALID_ARG;
    if (!it->second->done) return NTT_ERR_BUSY;
    srv->reqs.erase(it);
    return NTT_OK;
}

ntt_status ntt_server_stats_get(ntt_server* srv, ntt_server_stats* stats)
{
    if (!srv || !stats) return NTT_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(srv->mu);
    *stats = srv->stats;
    return NTT_OK;
}

}  // extern "C"

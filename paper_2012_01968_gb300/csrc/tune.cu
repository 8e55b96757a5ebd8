// Autotuner: times every compiled configuration of a transform size on the
// current device and keeps the fastest (the tuning parameters of Sec. VI-C,
// the radix split and the per-CTA tile, and of Sec. VII, the twiddle supply).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "host_logic.h"
#include "plan.h"

extern "C" void ntt_internal_set_cuda_error(cudaError_t e);

static_assert(NTT_KERNEL_AUTO == 0 && NTT_KERNEL_FUSED == 1 && NTT_KERNEL_PER_PASS == 2 && NTT_KERNEL_RADIX2 == 3 &&
                  NTT_KERNEL_HIGH_RADIX == 4 && NTT_KERNEL_CLUSTER == 5,
              "tune_candidates uses these codes");
static_assert(NTT_TWIDDLE_TABLE == 1 && NTT_TWIDDLE_OT == 2, "tune_candidates uses these codes");

namespace {

using Key = std::tuple<int, uint32_t, uint32_t, uint32_t, uint64_t>;   // device, N, L, batch, primes hash
std::mutex g_tune_mu;
std::map<Key, ntt_plan_opts> g_tune_cache;

uint64_t hash_primes(const uint64_t* primes, uint32_t L)
{
    uint64_t h = 0x9E3779B97F4A7C15ull;
    for (uint32_t i = 0; i < L; ++i) {
        h ^= primes[i] + 0x9E3779B97F4A7C15ull + (h << 6) + (h >> 2);
        h *= 0xBF58476D1CE4E5B9ull;
    }
    return h;
}

ntt_status cuda_fail(cudaError_t e)
{
    ntt_internal_set_cuda_error(e);
    return e == cudaErrorMemoryAllocation ? NTT_ERR_OOM : NTT_ERR_CUDA;
}

struct Scratch {
    std::vector<uint64_t*> bufs;
    cudaStream_t s = nullptr;
    cudaEvent_t ev[3] = {};
    ~Scratch()
    {
        for (uint64_t* b : bufs) cudaFree(b);
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
        if (s) cudaStreamDestroy(s);
    }
};

// Time one configuration; fills forward_us / inverse_us / status.
void time_one(ntt_tune_entry& r, uint32_t N, const uint64_t* primes, uint32_t L, uint32_t batch, uint32_t reps,
              Scratch& sc)
{
    ntt_plan* p = nullptr;
    r.status = ntt_plan_create(&p, N, primes, L, &r.opts);
    if (r.status != NTT_OK) return;
    const size_t nb = sc.bufs.size();
    ntt_status st = NTT_OK;
    for (int w = 0; w < 2 && st == NTT_OK; ++w) {
        st = ntt_forward(p, sc.bufs[w % nb], batch, sc.s);
        if (st == NTT_OK) st = ntt_inverse(p, sc.bufs[w % nb], batch, sc.s);
    }
    cudaError_t e = cudaEventRecord(sc.ev[0], sc.s);
    for (uint32_t i = 0; i < reps && st == NTT_OK; ++i) st = ntt_forward(p, sc.bufs[i % nb], batch, sc.s);
    if (e == cudaSuccess) e = cudaEventRecord(sc.ev[1], sc.s);
    for (uint32_t i = 0; i < reps && st == NTT_OK; ++i) st = ntt_inverse(p, sc.bufs[i % nb], batch, sc.s);
    if (e == cudaSuccess) e = cudaEventRecord(sc.ev[2], sc.s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(sc.s);
    float t1 = 0, t2 = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t1, sc.ev[0], sc.ev[1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t2, sc.ev[1], sc.ev[2]);
    uint32_t dev_status = 0;
    if (st == NTT_OK && e == cudaSuccess) st = ntt_plan_device_status(p, &dev_status);
    ntt_plan_destroy(p);
    if (st != NTT_OK) {
        r.status = st;
        return;
    }
    if (e != cudaSuccess) {
        r.status = cuda_fail(e);
        return;
    }
    if (dev_status != 0) {
        r.status = NTT_ERR_DEVICE;
        return;
    }
    r.forward_us = (double)t1 * 1e3 / reps;
    r.inverse_us = (double)t2 * 1e3 / reps;
}

}  // namespace

extern "C" ntt_status ntt_autotune(uint32_t N, const uint64_t* primes, uint32_t L, uint32_t batch, uint32_t reps,
                                   ntt_plan_opts* best, ntt_tune_entry* entries, uint32_t max_entries,
                                   uint32_t* count)
{
    if (!primes || !best || L == 0 || L > 4096 || batch == 0) return NTT_ERR_INVALID_ARG;
    if (N < 2 || N > (1u << 17) || (N & (N - 1))) return NTT_ERR_INVALID_ARG;
    if ((uint64_t)batch * L > 0xFFFFFFFFull) return NTT_ERR_INVALID_ARG;
    if (reps == 0) reps = 20;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    const Key key{dev, N, L, batch, hash_primes(primes, L)};
    if (!entries) {
        std::lock_guard<std::mutex> g(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            *best = it->second;
            if (count) *count = 0;
            return NTT_OK;
        }
    }
    const uint32_t n = (uint32_t)__builtin_ctz(N);
    const std::vector<ntt::host::TuneCandidate> cand =
        ntt::host::tune_candidates(n, (uint32_t)ntt::kGeometries, (uint32_t)ntt::SINGLE_PASS_MAX);

    // inputs: zero residues are canonical for every prime; enough buffers to
    // exceed twice the L2 between reuses, within 1 GiB
    Scratch sc;
    const size_t bytes = (size_t)batch * L * N * sizeof(uint64_t);
    int l2 = 0;
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
    size_t nbuf = (2 * (size_t)std::max(l2, 0)) / bytes + 1;
    nbuf = std::max<size_t>(1, std::min(nbuf, ((size_t)1 << 30) / std::max<size_t>(bytes, 1)));
    for (size_t i = 0; i < nbuf; ++i) {
        uint64_t* b = nullptr;
        e = cudaMalloc(&b, bytes);
        if (e != cudaSuccess) {
            if (i == 0) return cuda_fail(e);
            cudaGetLastError();
            break;
        }
        sc.bufs.push_back(b);
        e = cudaMemset(b, 0, bytes);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    e = cudaStreamCreateWithFlags(&sc.s, cudaStreamNonBlocking);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaEventCreate(&sc.ev[k]);
    if (e != cudaSuccess) return cuda_fail(e);

    std::vector<ntt_tune_entry> res(cand.size());
    std::vector<double> fw(cand.size()), iv(cand.size());
    std::vector<bool> ok(cand.size());
    for (size_t i = 0; i < cand.size(); ++i) {
        ntt_tune_entry& r = res[i];
        std::memset(&r, 0, sizeof(r));
        r.opts.kernel = cand[i].kernel;
        r.opts.twiddle_mode = cand[i].twiddle_mode;
        r.opts.ot_stages = cand[i].ot_stages;
        r.opts.geometry = cand[i].geometry;
        time_one(r, N, primes, L, batch, reps, sc);
        if (r.status == NTT_ERR_BAD_PRIME || r.status == NTT_ERR_CUDA) return r.status;
        fw[i] = r.forward_us;
        iv[i] = r.inverse_us;
        ok[i] = r.status == NTT_OK;
    }
    if (entries) {
        for (size_t i = 0; i < res.size() && i < max_entries; ++i) entries[i] = res[i];
    }
    if (count) *count = (uint32_t)res.size();
    const int b = ntt::host::tune_pick(fw, iv, ok);
    if (b < 0) return NTT_ERR_DEVICE;
    *best = res[(size_t)b].opts;
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune_cache[key] = *best;
    return NTT_OK;
}

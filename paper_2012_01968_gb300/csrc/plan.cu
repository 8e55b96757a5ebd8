// Plan creation: validate the primes, derive psi, build the device tables.
//
// Tables per prime q (paper: Sec. III-C Psi list, Algorithm 4 companions,
// Sec. VII on-the-fly twiddling):
//   tw[i]  = (Psi[i], floor(Psi[i] 2^64 / q)),  Psi[i] = psi^{brv(i)},  i < tw_len
//            (tw_len = N in table mode; 2^{n - ot} with OT, since the last ot
//            stages never read the table).  The inverse reads the same table:
//            Psi^{-1}[2^s + j] = -Psi[2^{s+1} - 1 - j].
//   OT factors of the second pass (s0 = p1 first stage, p2 stages):
//            Psi[2^s + (u << sl) + j] = A[2^sl + j] * B[sl][u],  s = s0 + sl,
//            A[2^sl + j] = psi^{2^{n-sl} brv_sl(j)},
//            B[sl][u]    = psi^{2^{n-1-s} (2 brv_s0(u) + 1)},
//            and the same with psi^{-1} for the inverse.
#include <cuda_runtime.h>

#include <cstring>
#include <new>
#include <thread>
#include <vector>

#include "numtheory.h"
#include "plan.h"

using ntt::Tw;
using ntt::PrimeDev;
namespace nt = ntt::nt;

extern "C" void ntt_internal_set_cuda_error(cudaError_t e);

// Make the fused kernel's work area cover `limbs` limbs (zero-filled).  A
// larger area replaces the old one after the device has drained.
cudaError_t ntt_internal_grow_work(ntt_plan* p, uint32_t limbs)
{
    std::lock_guard<std::mutex> g(p->work_mu);
    if (p->work_limbs >= limbs) return cudaSuccess;
    if (p->d_work) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return e;
        cudaFree(p->d_work);
        p->d_work = nullptr;
        p->work_limbs = 0;
    }
    const size_t bytes = ntt::fused_work_words(limbs) * sizeof(uint32_t);
    cudaError_t e = cudaMalloc(&p->d_work, bytes);
    if (e != cudaSuccess) return e;
    e = cudaMemset(p->d_work, 0, bytes);
    if (e != cudaSuccess) return e;
    p->work_limbs = limbs;
    return cudaSuccess;
}

namespace {

struct HostTables {
    std::vector<Tw> tw, ota_f, otb_f, ota_i, otb_i;
    std::vector<PrimeDev> pd;
};

Tw make_tw(uint64_t w, uint64_t q) { return Tw{w, nt::shoup_companion(w, q)}; }

void build_prime(const ntt_plan& p, uint32_t l, HostTables& h)
{
    const uint64_t q = p.primes[l], psi = p.psis[l];
    const uint32_t N = p.N, n = p.n;
    std::vector<uint64_t> pw(N);          // psi^e, e < N
    pw[0] = 1;
    for (uint32_t e = 1; e < N; ++e) pw[e] = nt::mulmod(pw[e - 1], psi, q);
    auto fwd = [&](uint64_t e) { return pw[e]; };                          // e < N
    auto inv = [&](uint64_t e) { return e == 0 ? 1 : q - pw[N - e]; };    // psi^{-e}, e < N

    // Psi[2^s + j] goes to slot 2^s + tw_slot(j) of the pass holding stage s
    // (natural order, slot 2^s + j, for the radix-2 organisation)
    Tw* tw = h.tw.data() + (size_t)l * p.tw_len;
    tw[0] = make_tw(1, q);
    const bool cluster = p.kernel == NTT_KERNEL_CLUSTER;
    for (uint32_t s = 0; (1u << s) < p.tw_len; ++s) {
        const ntt::StageSlot g = cluster ? ntt::stage_slot_params(n, p.p1, s, true, ntt::CLUSTER_TABLE_KMAX)
                                         : ntt::stage_slot_params(n, p.p1, s);
        for (uint32_t j = 0; j < (1u << s); ++j) {
            const bool natural = p.kernel == NTT_KERNEL_RADIX2 || p.kernel == NTT_KERNEL_HIGH_RADIX;
            const uint32_t slot = natural ? j : ntt::tw_slot(j, g.sl, g.K0, g.k);
            tw[(1u << s) + slot] = make_tw(fwd(nt::brv((1u << s) + j, n)), q);
        }
    }

    PrimeDev& d = h.pd[l];
    d.q = q;
    d.k = (uint32_t)nt::bitlen(q);
    d.mu = (uint64_t)(((nt::u128)1 << (2 * d.k)) / q);
    d.rc = (uint32_t)(((nt::u128)1 << (d.k + 31)) / q);   // < 2^32: q > 2^(k-1)
    d.rsh = d.k - 28;
    const uint64_t ninv = nt::powmod(N % q, q - 2, q);
    d.ninv = make_tw(ninv, q);
    const uint64_t psi_half = N >= 2 ? fwd(nt::brv(1, n)) : 1;   // Psi[1] = psi^{N/2}
    d.w1ninv = make_tw(nt::mulmod(psi_half, ninv, q), q);

    if (p.twiddle_mode == NTT_TWIDDLE_OT) {
        const uint32_t s0 = p.p1, p2 = n - p.p1, R = 1u << p2;
        Tw* af = h.ota_f.data() + (size_t)l * R;
        Tw* ai = h.ota_i.data() + (size_t)l * R;
        af[0] = ai[0] = make_tw(1, q);
        for (uint32_t sl = 0; sl < p2; ++sl) {
            const ntt::StageSlot g = ntt::stage_slot_params(n, p.p1, p.p1 + sl);
            for (uint32_t j = 0; j < (1u << sl); ++j) {
                const uint64_t e = ((uint64_t)nt::brv(j, sl)) << (n - sl);
                const uint32_t slot = (1u << sl) + ntt::tw_slot(j, g.sl, g.K0, g.k);
                af[slot] = make_tw(fwd(e), q);
                ai[slot] = make_tw(inv(e), q);
            }
        }
        const size_t bl = (size_t)p2 << s0;
        Tw* bf = h.otb_f.data() + (size_t)l * bl;
        Tw* bi = h.otb_i.data() + (size_t)l * bl;
        for (uint32_t sl = 0; sl < p2; ++sl)
            for (uint32_t u = 0; u < (1u << s0); ++u) {
                const uint32_t s = s0 + sl;
                const uint64_t e = ((uint64_t)(2 * nt::brv(u, s0) + 1)) << (n - 1 - s);
                bf[((size_t)sl << s0) + u] = make_tw(fwd(e), q);
                bi[((size_t)sl << s0) + u] = make_tw(inv(e), q);
            }
    }
}

template <class T>
cudaError_t upload(T** dst, const std::vector<T>& src, uint64_t& bytes)
{
    if (src.empty()) return cudaSuccess;
    const size_t sz = src.size() * sizeof(T);
    cudaError_t e = cudaMalloc(dst, sz);
    if (e != cudaSuccess) return e;
    bytes += sz;
    return cudaMemcpy(*dst, src.data(), sz, cudaMemcpyHostToDevice);
}

void free_plan(ntt_plan* p)
{
    if (!p) return;
    p->tables.reset();                  // frees the tables with the last plan sharing them
    cudaFree(p->d_stage);
    cudaFree(p->d_hwork);
    if (p->h_in) cudaStreamDestroy(p->h_in);
    if (p->h_out) cudaStreamDestroy(p->h_out);
    for (int k = 0; k < ntt_plan::kHostCompute; ++k)
        if (p->h_comp[k]) cudaStreamDestroy(p->h_comp[k]);
    if (p->hfork) cudaEventDestroy(p->hfork);
    if (p->h_join) cudaEventDestroy(p->h_join);
    for (int k = 0; k < ntt_plan::kHostSegments; ++k) {
        if (p->h_loaded[k]) cudaEventDestroy(p->h_loaded[k]);
        if (p->h_done[k]) cudaEventDestroy(p->h_done[k]);
        for (int b = 0; b < ntt_plan::kHostBuffers; ++b)
            if (p->h_out_done[b][k]) cudaEventDestroy(p->h_out_done[b][k]);
    }
    cudaFree(p->d_status);
    cudaFree(p->d_work);
    delete p;
}

// Persisting L2 for the twiddle table (NTT_PLAN_L2_TWIDDLES): raise this
// context's persisting-L2 limit to cover the table (never lower it), up to the
// device maximum, and keep the fraction of the window that fits.
std::mutex g_l2_mu;
cudaError_t reserve_l2(ntt_plan* p)
{
    const size_t bytes = (size_t)p->L * p->tw_len * sizeof(Tw);
    int max_persist = 0, max_window = 0;
    cudaError_t e = cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, p->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&max_window, cudaDevAttrMaxAccessPolicyWindowSize, p->device);
    if (e != cudaSuccess) return e;
    if (max_persist <= 0 || max_window <= 0 || bytes > (size_t)max_window) {
        p->l2_hit = 0.f;              // no window: the plan runs as without the flag
        return cudaSuccess;
    }
    std::lock_guard<std::mutex> g(g_l2_mu);
    size_t cur = 0;
    e = cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize);
    if (e != cudaSuccess) return e;
    const size_t want = std::min(bytes, (size_t)max_persist);
    if (cur < want) e = cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize);
    p->l2_hit = e == cudaSuccess ? (float)std::min(1.0, (double)cur / (double)bytes) : 0.f;
    return e;
}

}  // namespace

extern "C" ntt_status ntt_plan_create(ntt_plan** out, uint32_t N, const uint64_t* primes, uint32_t L,
                                      const ntt_plan_opts* opts)
{
    if (!out || !primes || L == 0 || L > 4096) return NTT_ERR_INVALID_ARG;
    if (N < 2 || N > (1u << 17) || (N & (N - 1))) return NTT_ERR_INVALID_ARG;
    ntt_plan_opts o;
    std::memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    if (o.reserved) return NTT_ERR_INVALID_ARG;
    if (o.flags & ~NTT_PLAN_L2_TWIDDLES) return NTT_ERR_INVALID_ARG;
    if (o.twiddle_mode > NTT_TWIDDLE_OT) return NTT_ERR_INVALID_ARG;
    if (o.kernel > NTT_KERNEL_CLUSTER) return NTT_ERR_INVALID_ARG;
    const bool high_radix = o.kernel == NTT_KERNEL_HIGH_RADIX;
    if (high_radix ? o.radix_log2 > 5 : o.radix_log2 != 0) return NTT_ERR_INVALID_ARG;
    if (o.geometry >= (uint32_t)ntt::kGeometries) return NTT_ERR_INVALID_ARG;
    if (o.ctas_per_sm > 8) return NTT_ERR_INVALID_ARG;
    const uint32_t n = (uint32_t)__builtin_ctz(N);
    const bool two_pass = n > (uint32_t)ntt::SINGLE_PASS_MAX;
    if (o.geometry && (!two_pass || o.kernel == NTT_KERNEL_RADIX2 || high_radix)) return NTT_ERR_INVALID_ARG;
    const bool cluster = o.kernel == NTT_KERNEL_CLUSTER;
    if (cluster && (n < (uint32_t)ntt::CLUSTER_N_MIN || n > (uint32_t)ntt::CLUSTER_N_MAX ||
                    o.twiddle_mode == NTT_TWIDDLE_OT || o.ot_stages))
        return NTT_ERR_INVALID_ARG;
    const uint32_t p1 = cluster    ? n / 2u
                        : two_pass ? (uint32_t)ntt::geometry_of((int)n, (int)o.geometry).p1
                                   : (uint32_t)ntt::split_p1((int)n);
    // AUTO: OT on the last stage for two-pass sizes (measured faster than the
    // table there, and half the last stage's twiddle traffic), table below
    const bool radix2 = o.kernel == NTT_KERNEL_RADIX2 || high_radix;   // global-memory organisations
    if (radix2 && o.twiddle_mode == NTT_TWIDDLE_OT) return NTT_ERR_INVALID_ARG;   // table twiddles only
    uint32_t mode = o.twiddle_mode;
    if (mode == NTT_TWIDDLE_AUTO) mode = two_pass && !radix2 ? NTT_TWIDDLE_OT : NTT_TWIDDLE_TABLE;
    uint32_t ots = 0;
    if (mode == NTT_TWIDDLE_OT) {
        ots = o.ot_stages ? o.ot_stages : 1;
        if (ots > 2) return NTT_ERR_INVALID_ARG;
        if (!two_pass) mode = NTT_TWIDDLE_TABLE, ots = 0;   // tables of <= 2^12 entries
    } else if (o.ot_stages) {
        return NTT_ERR_INVALID_ARG;
    }
    for (uint32_t l = 0; l < L; ++l) {
        const uint64_t q = primes[l];
        if (q <= (1ull << 32) || q >= (1ull << 60)) return NTT_ERR_BAD_PRIME;
        if ((q - 1) % (2ull * N) != 0) return NTT_ERR_BAD_PRIME;
        if (!nt::is_prime(q)) return NTT_ERR_BAD_PRIME;
    }

    ntt_plan* p = new (std::nothrow) ntt_plan();
    if (!p) return NTT_ERR_OOM;
    p->N = N;
    p->n = n;
    p->L = L;
    p->p1 = p1;
    p->passes = two_pass ? 2 : 1;
    p->twiddle_mode = mode;
    p->ot_stages = ots;
    p->kernel = cluster                            ? NTT_KERNEL_CLUSTER
                : high_radix                       ? NTT_KERNEL_HIGH_RADIX
                : radix2                           ? NTT_KERNEL_RADIX2
                : o.kernel == NTT_KERNEL_PER_PASS ? NTT_KERNEL_PER_PASS
                                                   : NTT_KERNEL_FUSED;
    p->radix_log2 = high_radix ? (o.radix_log2 ? o.radix_log2 : 4u) : 0u;
    p->geom = o.geometry;
    p->flags = o.flags;
    p->ctas_per_sm = o.ctas_per_sm;
    cudaError_t ce = cudaGetDevice(&p->device);
    if (ce != cudaSuccess) {
        ntt_internal_set_cuda_error(ce);
        delete p;
        return NTT_ERR_CUDA;
    }
    p->primes.assign(primes, primes + L);
    p->psis.resize(L);
    for (uint32_t l = 0; l < L; ++l) {
        const uint64_t q = primes[l];
        const uint64_t g = nt::smallest_generator(q);
        p->psis[l] = nt::powmod(g, (q - 1) / (2ull * N), q);
    }
    p->tw_len = N >> ots;

    HostTables h;
    try {
        h.tw.resize((size_t)L * p->tw_len);
        h.pd.resize(L);
        if (mode == NTT_TWIDDLE_OT) {
            const size_t R = (size_t)1 << (n - p1), bl = (size_t)(n - p1) << p1;
            h.ota_f.resize(L * R);
            h.ota_i.resize(L * R);
            h.otb_f.resize(L * bl);
            h.otb_i.resize(L * bl);
        }
    } catch (...) {
        delete p;
        return NTT_ERR_OOM;
    }
    const unsigned hw = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    const unsigned nth = std::min<unsigned>(hw, L);
    if (nth <= 1 || (size_t)N * L < (1u << 16)) {
        for (uint32_t l = 0; l < L; ++l) build_prime(*p, l, h);
    } else {
        std::vector<std::thread> th;
        for (unsigned t = 0; t < nth; ++t)
            th.emplace_back([&, t] {
                for (uint32_t l = t; l < L; l += nth) build_prime(*p, l, h);
            });
        for (auto& t : th) t.join();
    }

    ce = cudaMalloc(&p->d_status, sizeof(uint32_t));
    if (ce == cudaSuccess) ce = cudaMemset(p->d_status, 0, sizeof(uint32_t));
    if (ce == cudaSuccess) ce = ntt_internal_grow_work(p, L * 16u);
    p->tables = std::make_shared<NttPlanTables>();
    NttPlanTables& t = *p->tables;
    if (ce == cudaSuccess) ce = upload(&t.primes, h.pd, p->device_bytes);
    if (ce == cudaSuccess) ce = upload(&t.tw, h.tw, p->device_bytes);
    if (ce == cudaSuccess) ce = upload(&t.ota_f, h.ota_f, p->device_bytes);
    if (ce == cudaSuccess) ce = upload(&t.otb_f, h.otb_f, p->device_bytes);
    if (ce == cudaSuccess) ce = upload(&t.ota_i, h.ota_i, p->device_bytes);
    if (ce == cudaSuccess) ce = upload(&t.otb_i, h.otb_i, p->device_bytes);
    p->d_primes = t.primes;
    p->d_tw = t.tw;
    p->d_ota_f = t.ota_f;
    p->d_otb_f = t.otb_f;
    p->d_ota_i = t.ota_i;
    p->d_otb_i = t.otb_i;
    if (ce == cudaSuccess && (p->flags & NTT_PLAN_L2_TWIDDLES)) ce = reserve_l2(p);
    if (ce != cudaSuccess) {
        ntt_internal_set_cuda_error(ce);
        free_plan(p);
        cudaGetLastError();
        return ce == cudaErrorMemoryAllocation ? NTT_ERR_OOM : NTT_ERR_CUDA;
    }
    *out = p;
    return NTT_OK;
}

extern "C" void ntt_plan_destroy(ntt_plan* plan) { free_plan(plan); }

extern "C" ntt_status ntt_plan_set_ctas_per_sm(ntt_plan* p, uint32_t ctas_per_sm)
{
    if (!p || ctas_per_sm > 8) return NTT_ERR_INVALID_ARG;
    p->ctas_per_sm = ctas_per_sm;
    return NTT_OK;
}

extern "C" ntt_status ntt_plan_clone(ntt_plan** out, const ntt_plan* src)
{
    if (!out || !src) return NTT_ERR_INVALID_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != src->device) return NTT_ERR_INVALID_ARG;
    ntt_plan* p = new (std::nothrow) ntt_plan();
    if (!p) return NTT_ERR_OOM;
    p->N = src->N;
    p->n = src->n;
    p->L = src->L;
    p->p1 = src->p1;
    p->passes = src->passes;
    p->twiddle_mode = src->twiddle_mode;
    p->ot_stages = src->ot_stages;
    p->device = src->device;
    p->primes = src->primes;
    p->psis = src->psis;
    p->tables = src->tables;
    p->d_primes = src->d_primes;
    p->d_tw = src->d_tw;
    p->tw_len = src->tw_len;
    p->d_ota_f = src->d_ota_f;
    p->d_otb_f = src->d_otb_f;
    p->d_ota_i = src->d_ota_i;
    p->d_otb_i = src->d_otb_i;
    p->device_bytes = src->device_bytes;
    p->kernel = src->kernel;
    p->geom = src->geom;
    p->flags = src->flags;
    p->radix_log2 = src->radix_log2;
    p->ctas_per_sm = src->ctas_per_sm;
    p->l2_hit = src->l2_hit;
    cudaError_t ce = cudaMalloc(&p->d_status, sizeof(uint32_t));
    if (ce == cudaSuccess) ce = cudaMemset(p->d_status, 0, sizeof(uint32_t));
    if (ce == cudaSuccess) ce = ntt_internal_grow_work(p, src->work_limbs ? src->work_limbs : src->L * 16u);
    if (ce != cudaSuccess) {
        ntt_internal_set_cuda_error(ce);
        free_plan(p);
        cudaGetLastError();
        return ce == cudaErrorMemoryAllocation ? NTT_ERR_OOM : NTT_ERR_CUDA;
    }
    *out = p;
    return NTT_OK;
}

extern "C" ntt_status ntt_plan_query(const ntt_plan* p, ntt_plan_info* info)
{
    if (!p || !info) return NTT_ERR_INVALID_ARG;
    std::memset(info, 0, sizeof(*info));
    info->N = p->N;
    info->L = p->L;
    info->log2_N = p->n;
    info->passes = p->kernel == NTT_KERNEL_CLUSTER ? 2u : p->passes;
    info->pass1_log2 = p->p1;
    info->twiddle_mode = p->twiddle_mode;
    info->ot_stages = p->ot_stages;
    info->device = (uint32_t)p->device;
    info->kernel = p->kernel;
    info->device_bytes = p->device_bytes;
    info->geometry = p->geom;
    info->row_tile_log2 = p->passes == 2 ? (uint32_t)ntt::geometry_of((int)p->n, (int)p->geom).logc_r
                          : p->kernel == NTT_KERNEL_CLUSTER
                              ? p->p1 - (p->n - 9u)      // rows per CTA: 2^p1 rows over N / 512 CTAs
                              : 0;
    info->radix_log2 = p->radix_log2;
    info->ctas_per_sm = p->ctas_per_sm;
    return NTT_OK;
}

extern "C" ntt_status ntt_plan_device_status(const ntt_plan* p, uint32_t* status)
{
    if (!p || !status) return NTT_ERR_INVALID_ARG;
    cudaError_t e = cudaDeviceSynchronize();
    uint32_t v = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&v, p->d_status, sizeof(v), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(p->d_status, 0, sizeof(v));
    if (e != cudaSuccess) {
        ntt_internal_set_cuda_error(e);
        return NTT_ERR_CUDA;
    }
    *status = v;
    return NTT_OK;
}

extern "C" ntt_status ntt_plan_psi(const ntt_plan* p, uint32_t l, uint64_t* psi)
{
    if (!p || !psi || l >= p->L) return NTT_ERR_INVALID_ARG;
    *psi = p->psis[l];
    return NTT_OK;
}

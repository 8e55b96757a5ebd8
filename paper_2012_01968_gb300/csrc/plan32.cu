// 32-bit word plans (Sec. IV, "32b vs. 64b word size"): primes q < 2^28,
// residues in 32-bit words; the fused two-pass kernel for N >= 2^13 (table
// twiddles or OT of the last stage) or one launch per pass (table), one pass
// below.
//
// Tables per prime q, in the slot order of the 64-bit kernels (the pass split
// and the per-thread radix are the same):
//   tw[i] = (Psi[i], floor(Psi[i] 2^32 / q)),  Psi[i] = psi^{brv(i)},  i < tw_len
//   (N, or N / 2 when the last stage is twiddled on the fly from the OT
//   factors A and B of the 64-bit plans, in the same layout).
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "launch.cuh"
#include "numtheory.h"

namespace nt = ntt::nt;
using ntt::PrimeDev32;
using ntt::Tw32;

extern "C" void ntt_internal_set_cuda_error(cudaError_t e);

struct ntt_plan32 {
    uint32_t N = 0, n = 0, L = 0, p1 = 0;
    uint32_t kernel = 0;                  // NTT_KERNEL_FUSED or NTT_KERNEL_PER_PASS (two-pass sizes)
    uint32_t ots = 0;                     // stages twiddled on the fly (0 or 1, fused kernel)
    uint32_t tw_len = 0;                  // table entries per prime
    int device = 0;
    std::vector<uint32_t> primes, psis;
    PrimeDev32* d_primes = nullptr;
    Tw32* d_tw = nullptr;
    Tw32* d_ota_f = nullptr;              // OT factors, forward and inverse (ots > 0)
    Tw32* d_otb_f = nullptr;
    Tw32* d_ota_i = nullptr;
    Tw32* d_otb_i = nullptr;
    uint32_t* d_status = nullptr;         // device status word (fused kernel's bounded waits)
    uint32_t* d_work = nullptr;           // fused kernel's work area, fused_work_words(work_limbs) words
    uint32_t work_limbs = 0;
    std::mutex work_mu;
};

namespace {

Tw32 make_tw32(uint64_t w, uint64_t q) { return Tw32{(uint32_t)w, (uint32_t)((w << 32) / q)}; }

void free_plan32(ntt_plan32* p)
{
    if (!p) return;
    cudaFree(p->d_primes);
    cudaFree(p->d_tw);
    cudaFree(p->d_ota_f);
    cudaFree(p->d_otb_f);
    cudaFree(p->d_ota_i);
    cudaFree(p->d_otb_i);
    cudaFree(p->d_status);
    cudaFree(p->d_work);
    delete p;
}

// Make the work area cover `limbs` limbs (zero-filled); a larger area
// replaces the old one after the device has drained.
cudaError_t grow_work32(ntt_plan32* p, uint32_t limbs)
{
    std::lock_guard<std::mutex> g(p->work_mu);
    if (p->work_limbs >= limbs) return cudaSuccess;
    if (p->d_work) {
        const cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return e;
        cudaFree(p->d_work);
        p->d_work = nullptr;
        p->work_limbs = 0;
    }
    const size_t bytes = ntt::fused_work_words(limbs) * sizeof(uint32_t);
    cudaError_t e = cudaMalloc(&p->d_work, bytes);
    if (e == cudaSuccess) e = cudaMemset(p->d_work, 0, bytes);
    if (e == cudaSuccess) p->work_limbs = limbs;
    return e;
}

ntt_status to_status32(cudaError_t e)
{
    if (e == cudaSuccess) return NTT_OK;
    ntt_internal_set_cuda_error(e);
    return e == cudaErrorMemoryAllocation ? NTT_ERR_OOM : NTT_ERR_CUDA;
}

ntt_status transform32(const ntt_plan32* p, uint32_t* data, uint32_t batch, void* stream, bool fwd)
{
    if (!p || !data || batch == 0) return NTT_ERR_INVALID_ARG;
    if (((uintptr_t)data & 15u) != 0) return NTT_ERR_MISALIGNED;
    const uint64_t limbs = (uint64_t)batch * p->L;
    if (limbs > 0xFFFFFFFFull) return NTT_ERR_INVALID_ARG;
    if (p->n <= (uint32_t)ntt::SINGLE_PASS_MAX || p->kernel == NTT_KERNEL_PER_PASS) {
        const ntt::PassLaunch<ntt::u32> c{data, (uint32_t)limbs, p->L, p->n, p->d_primes, p->d_tw, p->tw_len,
                                          (cudaStream_t)stream};
        return to_status32(p->n <= (uint32_t)ntt::SINGLE_PASS_MAX ? ntt::launch_w32_single(c, fwd)
                                                                  : ntt::launch_w32_two(c, fwd));
    }
    if (limbs > 0x7FFFFFFFull) return NTT_ERR_INVALID_ARG;
    if (p->work_limbs < limbs) {
        const cudaError_t e = grow_work32(const_cast<ntt_plan32*>(p), (uint32_t)limbs);
        if (e != cudaSuccess) return to_status32(e);
    }
    const ntt::Fused32Launch c{data,      (uint32_t)limbs, p->L,         p->n,        p->d_primes,
                               p->d_tw,   p->tw_len,       p->d_status,   p->d_work,   p->work_limbs,
                               (cudaStream_t)stream,       p->ots,
                               fwd ? p->d_ota_f : p->d_ota_i, fwd ? p->d_otb_f : p->d_otb_i};
    return to_status32(ntt::launch_w32_fused(c, fwd));
}

}  // namespace

extern "C" ntt_status ntt_plan32_create(ntt_plan32** out, uint32_t N, const uint32_t* primes, uint32_t L,
                                        uint32_t kernel, uint32_t twiddle_mode)
{
    if (!out || !primes || L == 0 || L > 4096) return NTT_ERR_INVALID_ARG;
    if (kernel > NTT_KERNEL_PER_PASS || twiddle_mode > NTT_TWIDDLE_OT) return NTT_ERR_INVALID_ARG;
    if (N < 2 || N > (1u << 17) || (N & (N - 1))) return NTT_ERR_INVALID_ARG;
    const bool fused = N > (1u << ntt::SINGLE_PASS_MAX) && kernel != NTT_KERNEL_PER_PASS;
    if (twiddle_mode == NTT_TWIDDLE_OT && !fused) return NTT_ERR_INVALID_ARG;   // OT: fused two-pass plans only
    const uint32_t ots = fused && twiddle_mode != NTT_TWIDDLE_TABLE ? 1u : 0u;  // AUTO: OT1 where it applies
    for (uint32_t l = 0; l < L; ++l) {
        const uint64_t q = primes[l];
        if (q >= (1ull << 28)) return NTT_ERR_BAD_PRIME;       // 16 q must fit a word
        if ((q - 1) % (2ull * N) != 0 || q < 2) return NTT_ERR_BAD_PRIME;
        if (!nt::is_prime(q)) return NTT_ERR_BAD_PRIME;
    }
    ntt_plan32* p = new (std::nothrow) ntt_plan32();
    if (!p) return NTT_ERR_OOM;
    p->N = N;
    p->n = (uint32_t)__builtin_ctz(N);
    p->L = L;
    p->p1 = (uint32_t)ntt::split_p1((int)p->n);
    p->kernel = kernel == NTT_KERNEL_PER_PASS ? NTT_KERNEL_PER_PASS : NTT_KERNEL_FUSED;
    p->ots = ots;
    p->tw_len = N >> ots;
    cudaError_t ce = cudaGetDevice(&p->device);
    if (ce != cudaSuccess) {
        free_plan32(p);
        return to_status32(ce);
    }
    std::vector<Tw32> tw, ota_f, ota_i, otb_f, otb_i;
    std::vector<PrimeDev32> pd;
    const uint32_t p2 = p->n - p->p1;
    try {
        p->primes.assign(primes, primes + L);
        p->psis.resize(L);
        tw.resize((size_t)L * p->tw_len);
        pd.resize(L);
        if (ots) {
            ota_f.resize((size_t)L << p2);
            ota_i.resize((size_t)L << p2);
            otb_f.resize((size_t)L * ((size_t)p2 << p->p1));
            otb_i.resize((size_t)L * ((size_t)p2 << p->p1));
        }
    } catch (...) {
        free_plan32(p);
        return NTT_ERR_OOM;
    }
    const uint32_t n = p->n;
    std::vector<uint64_t> pw(N);
    for (uint32_t l = 0; l < L; ++l) {
        const uint64_t q = primes[l];
        const uint64_t psi = nt::powmod(nt::smallest_generator(q), (q - 1) / (2ull * N), q);
        p->psis[l] = (uint32_t)psi;
        pw[0] = 1;
        for (uint32_t e = 1; e < N; ++e) pw[e] = pw[e - 1] * psi % q;     // q < 2^28: no overflow
        auto inv = [&](uint64_t e) { return e == 0 ? 1 : q - pw[N - e]; };     // psi^{-e}, e < N
        Tw32* t = tw.data() + (size_t)l * p->tw_len;
        t[0] = make_tw32(1, q);
        for (uint32_t s = 0; (1u << s) < p->tw_len; ++s) {
            const ntt::StageSlot g = ntt::stage_slot_params((int)n, (int)p->p1, (int)s);
            for (uint32_t j = 0; j < (1u << s); ++j)
                t[(1u << s) + ntt::tw_slot(j, g.sl, g.K0, g.k)] = make_tw32(pw[nt::brv((1u << s) + j, n)], q);
        }
        if (ots) {
            // OT factors of the second pass (stages s0 + sl, s0 = p1):
            // Psi[2^s + (u << sl) + j] = A[2^sl + j] * B[sl][u]
            const uint32_t s0 = p->p1, R = 1u << p2;
            Tw32* af = ota_f.data() + (size_t)l * R;
            Tw32* ai = ota_i.data() + (size_t)l * R;
            af[0] = ai[0] = make_tw32(1, q);
            for (uint32_t sl = 0; sl < p2; ++sl) {
                const ntt::StageSlot g = ntt::stage_slot_params((int)n, (int)s0, (int)(s0 + sl));
                for (uint32_t j = 0; j < (1u << sl); ++j) {
                    const uint64_t e = ((uint64_t)nt::brv(j, (int)sl)) << (n - sl);
                    const uint32_t slot = (1u << sl) + ntt::tw_slot(j, g.sl, g.K0, g.k);
                    af[slot] = make_tw32(pw[e], q);
                    ai[slot] = make_tw32(inv(e), q);
                }
            }
            const size_t bl = (size_t)p2 << s0;
            Tw32* bf = otb_f.data() + (size_t)l * bl;
            Tw32* bi = otb_i.data() + (size_t)l * bl;
            for (uint32_t sl = 0; sl < p2; ++sl)
                for (uint32_t u = 0; u < (1u << s0); ++u) {
                    const uint32_t s = s0 + sl;
                    const uint64_t e = ((uint64_t)(2 * nt::brv(u, (int)s0) + 1)) << (n - 1 - s);
                    bf[((size_t)sl << s0) + u] = make_tw32(pw[e], q);
                    bi[((size_t)sl << s0) + u] = make_tw32(inv(e), q);
                }
        }
        PrimeDev32& d = pd[l];
        d.q = (uint32_t)q;
        d.rc = 0;
        d.rsh = 0;
        d.k = (uint32_t)nt::bitlen(q);
        const uint64_t ninv = nt::powmod(N % q, q - 2, q);
        d.ninv = make_tw32(ninv, q);
        d.w1ninv = make_tw32(pw[nt::brv(1, n)] * ninv % q, q);     // Psi[1] N^{-1}
    }
    ce = cudaMalloc(&p->d_status, sizeof(uint32_t));
    if (ce == cudaSuccess) ce = cudaMemset(p->d_status, 0, sizeof(uint32_t));
    if (ce == cudaSuccess) ce = cudaMalloc(&p->d_primes, pd.size() * sizeof(PrimeDev32));
    if (ce == cudaSuccess) ce = cudaMemcpy(p->d_primes, pd.data(), pd.size() * sizeof(PrimeDev32), cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMalloc(&p->d_tw, tw.size() * sizeof(Tw32));
    if (ce == cudaSuccess) ce = cudaMemcpy(p->d_tw, tw.data(), tw.size() * sizeof(Tw32), cudaMemcpyHostToDevice);
    auto upload = [&](Tw32** dst, const std::vector<Tw32>& src) {
        if (ce != cudaSuccess || src.empty()) return;
        ce = cudaMalloc(dst, src.size() * sizeof(Tw32));
        if (ce == cudaSuccess) ce = cudaMemcpy(*dst, src.data(), src.size() * sizeof(Tw32), cudaMemcpyHostToDevice);
    };
    upload(&p->d_ota_f, ota_f);
    upload(&p->d_ota_i, ota_i);
    upload(&p->d_otb_f, otb_f);
    upload(&p->d_otb_i, otb_i);
    if (ce != cudaSuccess) {
        free_plan32(p);
        cudaGetLastError();
        return to_status32(ce);
    }
    *out = p;
    return NTT_OK;
}

extern "C" void ntt_plan32_destroy(ntt_plan32* plan) { free_plan32(plan); }

extern "C" ntt_status ntt_forward32(const ntt_plan32* p, uint32_t* data, uint32_t batch, void* stream)
{
    return transform32(p, data, batch, stream, true);
}

extern "C" ntt_status ntt_inverse32(const ntt_plan32* p, uint32_t* data, uint32_t batch, void* stream)
{
    return transform32(p, data, batch, stream, false);
}

extern "C" ntt_status ntt_plan32_device_status(const ntt_plan32* p, uint32_t* status)
{
    if (!p || !status) return NTT_ERR_INVALID_ARG;
    cudaError_t e = cudaDeviceSynchronize();
    uint32_t v = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&v, p->d_status, sizeof(v), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(p->d_status, 0, sizeof(v));
    if (e != cudaSuccess) return to_status32(e);
    *status = v;
    return NTT_OK;
}

extern "C" ntt_status ntt_plan32_psi(const ntt_plan32* p, uint32_t l, uint32_t* psi)
{
    if (!p || !psi || l >= p->L) return NTT_ERR_INVALID_ARG;
    *psi = p->psis[l];
    return NTT_OK;
}

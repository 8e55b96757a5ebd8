// ntt_transform_noalloc: a transform call that allocates nothing, for callers
// that may not allocate device memory while they run (see the header).  The
// paper has no counterpart; this is a library interface.
//
// The only per-call scratch of the transform is the work area of the one-launch
// two-pass kernel (N >= 2^13): 4 + 2 * limbs 32-bit words that must all be
// zero when a launch starts and that the launch's last CTA zeroes again before
// it exits.  Here that area is a file-scope __device__ array, sized for
// NTT_NOALLOC_MAX_LIMBS limbs (64 KB).  The CUDA runtime zero-initialises it when
// it loads this module on a device, so the zero-at-start condition holds for the
// first launch and every completed launch restores it.  The kernel itself is the
// same one the plan's own entry points launch; only the work area differs.
//
// Each device has its own copy of the array.  Its address is looked up once
// per device (cudaGetSymbolAddress, with that device current) and cached; that
// first call may load the module, so it belongs before any stream capture.
// All calls on one device share the one area, so calls that overlap in time
// (two streams, two host threads, two plans) race on it.
#include <atomic>
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "plan.h"

extern "C" void ntt_internal_set_cuda_error(cudaError_t e);

static __device__ __align__(256) uint32_t g_noalloc_work[ntt::fused_work_words(NTT_NOALLOC_MAX_LIMBS)];

namespace {

constexpr int kMaxDevices = 64;
std::atomic<uint32_t*> g_work[kMaxDevices];
std::mutex g_setup_mu;

// Address of this device's copy of the work area; set-up on first use.
ntt_status noalloc_work(int device, uint32_t** out)
{
    if (device < 0 || device >= kMaxDevices) return NTT_ERR_INVALID_ARG;
    uint32_t* w = g_work[device].load(std::memory_order_acquire);
    if (!w) {
        std::lock_guard<std::mutex> g(g_setup_mu);
        w = g_work[device].load(std::memory_order_relaxed);
        if (!w) {
            void* addr = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_work);
            if (e != cudaSuccess || !addr) {
                ntt_internal_set_cuda_error(e != cudaSuccess ? e : cudaErrorInvalidSymbol);
                cudaGetLastError();
                return NTT_ERR_CUDA;
            }
            w = static_cast<uint32_t*>(addr);
            g_work[device].store(w, std::memory_order_release);
        }
    }
    *out = w;
    return NTT_OK;
}

}  // namespace

extern "C" ntt_status ntt_transform_noalloc(const ntt_plan* p, uint64_t* data, uint32_t batch,
                                            uint32_t levels, uint32_t op, void* stream)
{
    if (!p || !data || batch == 0 || levels == 0 || levels > p->L) return NTT_ERR_INVALID_ARG;
    if (op != NTT_OP_FORWARD && op != NTT_OP_INVERSE) return NTT_ERR_INVALID_ARG;
    if (((uintptr_t)data & 15u) != 0) return NTT_ERR_MISALIGNED;
    const uint64_t limbs = (uint64_t)batch * levels;
    if (limbs > NTT_NOALLOC_MAX_LIMBS) return NTT_ERR_LIMIT;
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        ntt_internal_set_cuda_error(e);
        return NTT_ERR_CUDA;
    }
    if (dev != p->device) return NTT_ERR_INVALID_ARG;
    uint32_t* work = nullptr;
    const ntt_status st = noalloc_work(dev, &work);
    if (st != NTT_OK) return st;
    ntt::LaunchCtx c = p->ctx(data, (uint32_t)limbs, levels, (cudaStream_t)stream);
    c.work = work;
    c.work_limbs = NTT_NOALLOC_MAX_LIMBS;
    e = ntt::launch_transform(c, op == NTT_OP_FORWARD);
    if (e != cudaSuccess) {
        ntt_internal_set_cuda_error(e);
        return NTT_ERR_CUDA;
    }
    return NTT_OK;
}

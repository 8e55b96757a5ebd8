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
// Each device has its own copy of the array, and each CUDA context on that
// device (the primary context is destroyed by cudaDeviceReset and made again
// later; a caller may also switch to a context of its own) loads the module
// anew, at a new address.  The address is therefore looked up
// (cudaGetSymbolAddress, with that device current) and cached per device
// together with the unique id of the context it belongs to; a call under
// another context looks it up again.  A look-up may load the module, so the
// first call in each context belongs before any stream capture.  All calls in
// one context share the one area, so calls that overlap in time (two streams,
// two host threads, two plans) race on it.
#include <cstdint>
#include <mutex>

#include <cuda.h>
#include <cuda_runtime.h>

#include "plan.h"

extern "C" void ntt_internal_set_cuda_error(cudaError_t e);

static __device__ __align__(256) uint32_t g_noalloc_work[ntt::fused_work_words(NTT_NOALLOC_MAX_LIMBS)];

namespace {

constexpr int kMaxDevices = 64;
struct Cached {
    unsigned long long ctx_id = 0;    // 0: none (context ids start at 1)
    uint32_t* addr = nullptr;
};
Cached g_work[kMaxDevices];
std::mutex g_mu;

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

// Unique id of the calling thread's current context (0 if it cannot be read).
unsigned long long current_context_id()
{
    static std::once_flag once;
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(p);
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// Address of the current context's copy of the work area on `device`.
ntt_status noalloc_work(int device, uint32_t** out)
{
    if (device < 0 || device >= kMaxDevices) return NTT_ERR_INVALID_ARG;
    const unsigned long long id = current_context_id();
    std::lock_guard<std::mutex> g(g_mu);
    Cached& c = g_work[device];
    if (id == 0 || c.ctx_id != id || !c.addr) {
        void* addr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_work);
        if (e != cudaSuccess || !addr) {
            ntt_internal_set_cuda_error(e != cudaSuccess ? e : cudaErrorInvalidSymbol);
            cudaGetLastError();
            return NTT_ERR_CUDA;
        }
        c.addr = static_cast<uint32_t*>(addr);
        c.ctx_id = id;
    }
    *out = c.addr;
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

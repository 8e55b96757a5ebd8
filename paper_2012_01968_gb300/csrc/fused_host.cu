// Host helpers for the fused launch: tensor maps and per-launch scratch.
#include <atomic>
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "plan.h"

namespace ntt {

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

cudaError_t encode_2d(CUtensorMap* m, void* base, uint64_t inner, uint64_t outer, uint64_t row_bytes,
                      uint32_t box_inner, uint32_t box_outer, CUtensorMapDataType type = CU_TENSOR_MAP_DATA_TYPE_UINT64)
{
    auto fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    const cuuint64_t dims[2] = {inner, outer};
    const cuuint64_t strides[1] = {row_bytes};
    const cuuint32_t box[2] = {box_inner, box_outer};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = fn(m, type, 2, base, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

// Column view: [N1 * limbs rows][N2 words], box 16 words x R1 rows.
// Row view:    [N / 16 * limbs lines][16 words], box 16 words x row_tile/16 lines.
cudaError_t encode_tile_maps(u64* data, u32 limbs, u32 n, int p1, int row_tile_words, CUtensorMap* mapC,
                             CUtensorMap* mapR)
{
    const uint64_t N = 1ull << n, N1 = 1ull << p1, N2 = N >> p1;
    cudaError_t e = encode_2d(mapC, data, N2, N1 * limbs, N2 * 8, 16, (uint32_t)N1);
    if (e != cudaSuccess) return e;
    return encode_2d(mapR, data, 16, (N / 16) * limbs, 128, 16, (uint32_t)(row_tile_words / 16));
}

// The same views of 32-bit words: 128-byte lines of 32 words.
cudaError_t encode_tile_maps32(u32* data, u32 limbs, u32 n, int p1, int row_tile_words, CUtensorMap* mapC,
                               CUtensorMap* mapR)
{
    const uint64_t N = 1ull << n, N1 = 1ull << p1, N2 = N >> p1;
    cudaError_t e = encode_2d(mapC, data, N2, N1 * limbs, N2 * 4, 32, (uint32_t)N1, CU_TENSOR_MAP_DATA_TYPE_UINT32);
    if (e != cudaSuccess) return e;
    return encode_2d(mapR, data, 32, (N / 32) * limbs, 128, 32, (uint32_t)(row_tile_words / 32),
                     CU_TENSOR_MAP_DATA_TYPE_UINT32);
}

namespace {

// SM count and L2 size of a device, queried once per device
struct DevAttrs {
    std::atomic<int> sms{0}, l2{0};
};
DevAttrs g_attrs[64];

const DevAttrs& attrs()
{
    int dev = 0;
    cudaGetDevice(&dev);
    DevAttrs& a = g_attrs[dev >= 0 && dev < 64 ? dev : 0];
    if (a.sms.load(std::memory_order_relaxed) == 0) {
        int sms = 0, l2 = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
        a.l2.store(l2 > 0 ? l2 : (32 << 20), std::memory_order_relaxed);
        a.sms.store(sms > 0 ? sms : 1, std::memory_order_release);
    }
    return a;
}

}  // namespace

int device_sm_count() { return attrs().sms.load(std::memory_order_acquire); }

}  // namespace ntt
